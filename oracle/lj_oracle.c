/*
 * lj_oracle.c -- plain, slow, FP64 CPU oracle for the Lennard-Jones MD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this file: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg use it.  It shares no code, header, table or helper with the CUDA
 * library in paper_1308_5587_gb300/csrc and includes nothing from it.
 *
 * What it computes (HOOMD-blue paper, Section 3.1 "Molecular dynamics" and
 * Listing 1: particles in a periodic box, md.nlist.cell + md.pair.lj(r_cut) with
 * pair_coeff epsilon/sigma, NVE among the listed ensembles, run(n); Section 7.1:
 * the LJ unit test checks "force, energy and virial").  The paper prints no
 * equations, so every formula below is the textbook definition; each reading the
 * paper leaves open is marked "paper silent":
 *
 *  - minimum image (paper silent):  d = x_i - x_j;  d <- d - L * rint(d / L)
 *    per axis, rint = round half to even.
 *  - energy-shifted, truncated 12-6 LJ (shift mode paper silent):
 *      V(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] - V_LJ(r_cut)   for r < r_cut
 *      V(r) = 0                                                   otherwise
 *    force on i from j:  F_ij = 24 eps [2 (sigma/r)^12 - (sigma/r)^6] / r^2 * d_ij
 *    (the force is not shifted).
 *  - the other short-range pair potentials named with LJ in Section 3.1 ("Mie,
 *    WCA, Yukawa, Gaussian"; the paper gives no formulas, these are their
 *    textbook forms), each truncated at r_cut and shifted by its value there,
 *    the force not shifted (kind codes as in the C library's interface):
 *      1 Mie(n, m):  V = C eps [(sigma/r)^n - (sigma/r)^m],
 *                    C = n/(n-m) (n/m)^(m/(n-m))  (so min V = -eps);
 *                    f = C eps [n (sigma/r)^n - m (sigma/r)^m] / r^2
 *      2 WCA:        12-6 LJ cut at its minimum, r_cut = 2^(1/6) sigma whatever
 *                    the rcut table says, so V = 4 eps [...] + eps >= 0
 *      3 Yukawa(kappa): V = eps exp(-kappa r) / r;
 *                    f = eps exp(-kappa r) (1 + kappa r) / r^3
 *      4 Gaussian:   V = eps exp(-r^2 / (2 sigma^2));  f = eps / sigma^2 exp(...)
 *    with F_ij = f d_ij as for LJ.  Mie takes n, m and Yukawa kappa from two
 *    extra per type-pair tables (pa, pb).
 *  - totals: F_i = sum_{j != i} F_ij;  U = sum_{i<j} V(r_ij);
 *    virial tensor W_ab = sum_{i<j} d_ij,a F_ij,b, stored xx,xy,xz,yy,yz,zz;
 *    per-particle energy and virial take half of every pair they are in.
 *  - kinetics: K = 1/2 m sum v^2,  T = 2K / (3N - 3),  P = (N T + tr(W)/3) / V
 *    (degrees of freedom and pressure form: paper silent).
 *  - velocity Verlet (NVE; the scheme itself is paper silent):
 *      v += dt/(2m) F;  x += dt v;  wrap;  F = F(x);  v += dt/(2m) F.
 *  - wrap (paper silent): centred box [-L/2, L/2): k = floor((x + L/2)/L),
 *    x -= k L, image += k.
 *  - reference neighbour set: every unordered pair i<j with min-image
 *    r^2 < (r_cut,ij + r_buff)^2, by brute force.
 *
 * Every loop is O(N^2) on purpose.  OpenMP only splits the outer i loop; every
 * per-particle sum runs over j in ascending order and every total is summed in
 * ascending i afterwards, so results do not depend on the thread count.
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 0; /* 0 = OpenMP default */

void oracle_set_threads(int n) { g_threads = n; }

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* minimum-image component (paper silent; textbook periodic boundary) */
static double min_image(double d, double L) { return d - L * rint(d / L); }

/* Truncated, energy-shifted LJ for one pair type at squared distance r2 < rc^2.
 * Writes the pair energy and the scalar f such that F_ij = f * d_ij. */
static void lj_pair(double r2, double eps, double sigma, double rc, double *v, double *f)
{
    double s2 = sigma * sigma / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    double c2 = sigma * sigma / (rc * rc);
    double c6 = c2 * c2 * c2;
    double c12 = c6 * c6;
    double v_at_cut = 4.0 * eps * (c12 - c6);
    *v = 4.0 * eps * (s12 - s6) - v_at_cut;
    *f = 24.0 * eps * (2.0 * s12 - s6) / r2;
}

enum { POT_LJ = 0, POT_MIE = 1, POT_WCA = 2, POT_YUKAWA = 3, POT_GAUSS = 4, POT_COUNT = 5 };

/* the pair interaction: which potential, and its per type-pair tables */
typedef struct {
    int32_t ntypes, kind;
    const double *eps, *sigma, *rcut, *pa, *pb;
} pair_model;

/* the cut-off radius of type pair p (WCA: the LJ minimum) */
static double cut_of(const pair_model *m, int32_t p)
{
    if (m->kind == POT_WCA) return pow(2.0, 1.0 / 6.0) * m->sigma[p];
    return m->rcut[p];
}

/* unshifted Mie energy and f at squared distance r2 */
static void mie_raw(double r2, double eps, double sigma, double n, double m, double *v, double *f)
{
    double c = n / (n - m) * pow(n / m, m / (n - m));
    double sn = pow(sigma * sigma / r2, 0.5 * n); /* (sigma/r)^n */
    double sm = pow(sigma * sigma / r2, 0.5 * m);
    *v = c * eps * (sn - sm);
    *f = c * eps * (n * sn - m * sm) / r2;
}

/* unshifted Yukawa energy and f at squared distance r2 */
static void yukawa_raw(double r2, double eps, double kappa, double *v, double *f)
{
    double r = sqrt(r2);
    double e = eps * exp(-kappa * r) / r;
    *v = e;
    *f = e * (1.0 + kappa * r) / r2;
}

/* unshifted Gaussian energy and f at squared distance r2 */
static void gauss_raw(double r2, double eps, double sigma, double *v, double *f)
{
    double e = eps * exp(-r2 / (2.0 * sigma * sigma));
    *v = e;
    *f = e / (sigma * sigma);
}

/* The pair interaction of type pair p at squared distance r2 < rc^2: energy shifted
 * by its value at rc, unshifted force factor f (F_ij = f d_ij). */
static void pair_terms(const pair_model *m, int32_t p, double r2, double rc, double *v, double *f)
{
    double vc, fc;
    switch (m->kind) {
    case POT_MIE:
        mie_raw(r2, m->eps[p], m->sigma[p], m->pa[p], m->pb[p], v, f);
        mie_raw(rc * rc, m->eps[p], m->sigma[p], m->pa[p], m->pb[p], &vc, &fc);
        *v -= vc;
        break;
    case POT_YUKAWA:
        yukawa_raw(r2, m->eps[p], m->pa[p], v, f);
        yukawa_raw(rc * rc, m->eps[p], m->pa[p], &vc, &fc);
        *v -= vc;
        break;
    case POT_GAUSS:
        gauss_raw(r2, m->eps[p], m->sigma[p], v, f);
        gauss_raw(rc * rc, m->eps[p], m->sigma[p], &vc, &fc);
        *v -= vc;
        break;
    default: /* LJ, and WCA with its own rc */
        lj_pair(r2, m->eps[p], m->sigma[p], rc, v, f);
    }
}

/* All interactions of particle i (j runs over every other particle, ascending).
 * Outputs the force on i, half of its pair energies and half of its pair virials. */
static void particle_terms(int64_t i, int64_t n, const double *box, const double *pos,
                           const int32_t *type, const pair_model *m, double f_out[3],
                           double *u_out, double w_out[6])
{
    double fx = 0, fy = 0, fz = 0, u = 0;
    double w[6] = {0, 0, 0, 0, 0, 0};
    int32_t ti = type[i];
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double dx = min_image(pos[3 * i + 0] - pos[3 * j + 0], box[0]);
        double dy = min_image(pos[3 * i + 1] - pos[3 * j + 1], box[1]);
        double dz = min_image(pos[3 * i + 2] - pos[3 * j + 2], box[2]);
        double r2 = dx * dx + dy * dy + dz * dz;
        int32_t p = ti * m->ntypes + type[j];
        double rc = cut_of(m, p);
        if (!(r2 < rc * rc)) continue;
        double v, f;
        pair_terms(m, p, r2, rc, &v, &f);
        fx += f * dx;
        fy += f * dy;
        fz += f * dz;
        u += 0.5 * v;
        w[0] += 0.5 * dx * (f * dx);
        w[1] += 0.5 * dx * (f * dy);
        w[2] += 0.5 * dx * (f * dz);
        w[3] += 0.5 * dy * (f * dy);
        w[4] += 0.5 * dy * (f * dz);
        w[5] += 0.5 * dz * (f * dz);
    }
    f_out[0] = fx;
    f_out[1] = fy;
    f_out[2] = fz;
    *u_out = u;
    for (int a = 0; a < 6; ++a) w_out[a] = w[a];
}

static int check_common(int64_t n, const double *box, int32_t ntypes)
{
    if (n < 0 || ntypes < 1 || !box) return -1;
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0)) return -1;
    return 0;
}

/* the pair model of the arguments, or -1 if a table its kind needs is missing */
static int make_model(pair_model *m, int32_t ntypes, int32_t kind, const double *eps,
                      const double *sigma, const double *rcut, const double *pa,
                      const double *pb)
{
    m->ntypes = ntypes;
    m->kind = kind;
    m->eps = eps;
    m->sigma = sigma;
    m->rcut = rcut;
    m->pa = pa;
    m->pb = pb;
    if (kind < 0 || kind >= POT_COUNT || !eps) return -1;
    if (kind != POT_YUKAWA && !sigma) return -1;
    if (kind != POT_WCA && !rcut) return -1;
    if ((kind == POT_MIE && (!pa || !pb)) || (kind == POT_YUKAWA && !pa)) return -1;
    return 0;
}

/* the same model with every entry's cut-off resolved (cut_of) into rc_out */
static void resolved_cuts(const pair_model *m, double *rc_out)
{
    for (int32_t p = 0; p < m->ntypes * m->ntypes; ++p) rc_out[p] = cut_of(m, p);
}

static int forces_model(int64_t n, const double *box, const double *pos, const int32_t *type,
                        const pair_model *m, double *force, double *energy, double *virial,
                        double *per_energy, double *per_virial);

/*
 * Forces, total potential energy and virial tensor of the whole system.
 * pos: n x 3 row-major, any image.  eps/sigma/rcut: ntypes x ntypes row-major.
 * force: n x 3 out.  energy: scalar out.  virial: 6 out (xx,xy,xz,yy,yz,zz).
 * per_energy / per_virial: optional (NULL) per-particle halves (n, n x 6).
 */
int oracle_forces(int64_t n, const double *box, const double *pos, const int32_t *type,
                  int32_t ntypes, int32_t kind, const double *eps, const double *sigma,
                  const double *rcut, const double *pa, const double *pb, double *force,
                  double *energy, double *virial, double *per_energy, double *per_virial)
{
    pair_model m;
    if (check_common(n, box, ntypes) || make_model(&m, ntypes, kind, eps, sigma, rcut, pa, pb))
        return -1;
    return forces_model(n, box, pos, type, &m, force, energy, virial, per_energy, per_virial);
}

static int forces_model(int64_t n, const double *box, const double *pos, const int32_t *type,
                        const pair_model *m, double *force, double *energy, double *virial,
                        double *per_energy, double *per_virial)
{
    double *u = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *w = (double *)malloc(sizeof(double) * 6 * (size_t)(n > 0 ? n : 1));
    if (!u || !w) {
        free(u);
        free(w);
        return -2;
    }
#pragma omp parallel for schedule(dynamic, 16) num_threads(oracle_get_threads())
    for (int64_t i = 0; i < n; ++i)
        particle_terms(i, n, box, pos, type, m, &force[3 * i], &u[i], &w[6 * i]);
    double U = 0, W[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        U += u[i];
        for (int a = 0; a < 6; ++a) W[a] += w[6 * i + a];
    }
    if (energy) *energy = U;
    if (virial)
        for (int a = 0; a < 6; ++a) virial[a] = W[a];
    if (per_energy) memcpy(per_energy, u, sizeof(double) * (size_t)n);
    if (per_virial) memcpy(per_virial, w, sizeof(double) * 6 * (size_t)n);
    free(u);
    free(w);
    return 0;
}

/*
 * The same per-particle quantities for a listed subset of particles only
 * (cost O(m n)); used to check sampled outputs of systems too large for O(n^2).
 */
int oracle_forces_subset(int64_t n, const double *box, const double *pos, const int32_t *type,
                         int32_t ntypes, int32_t kind, const double *eps, const double *sigma,
                         const double *rcut, const double *pa, const double *pb, int64_t m,
                         const int64_t *idx, double *force, double *per_energy,
                         double *per_virial)
{
    pair_model pm;
    if (check_common(n, box, ntypes) || m < 0 ||
        make_model(&pm, ntypes, kind, eps, sigma, rcut, pa, pb))
        return -1;
    for (int64_t k = 0; k < m; ++k)
        if (idx[k] < 0 || idx[k] >= n) return -1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(oracle_get_threads())
    for (int64_t k = 0; k < m; ++k) {
        double u, w[6];
        particle_terms(idx[k], n, box, pos, type, &pm, &force[3 * k], &u, w);
        if (per_energy) per_energy[k] = u;
        if (per_virial)
            for (int a = 0; a < 6; ++a) per_virial[6 * k + a] = w[a];
    }
    return 0;
}

/*
 * Reference neighbour set (paper: md.nlist.cell builds it; the skin r_buff and the
 * strict '<' are paper silent): all pairs i<j with r^2 < rlist_ij^2, ascending in
 * (i, j).  Writes at most cap pairs (pairs: cap x 2, r: cap) and returns the total
 * count in *npairs (which may exceed cap: call again with more room).
 */
int oracle_neighbors(int64_t n, const double *box, const double *pos, const int32_t *type,
                     int32_t ntypes, const double *rlist, int64_t cap, int32_t *pairs,
                     double *r, int64_t *npairs)
{
    if (check_common(n, box, ntypes) || cap < 0 || !npairs) return -1;
    int64_t *cnt = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    if (!cnt) return -2;
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(oracle_get_threads())
        for (int64_t i = 0; i < n; ++i) {
            int64_t c = 0, out = pass ? cnt[i] : 0;
            for (int64_t j = i + 1; j < n; ++j) {
                double dx = min_image(pos[3 * i + 0] - pos[3 * j + 0], box[0]);
                double dy = min_image(pos[3 * i + 1] - pos[3 * j + 1], box[1]);
                double dz = min_image(pos[3 * i + 2] - pos[3 * j + 2], box[2]);
                double r2 = dx * dx + dy * dy + dz * dz;
                double rl = rlist[type[i] * ntypes + type[j]];
                if (!(r2 < rl * rl)) continue;
                if (pass && out + c < cap) {
                    pairs[2 * (out + c) + 0] = (int32_t)i;
                    pairs[2 * (out + c) + 1] = (int32_t)j;
                    if (r) r[out + c] = sqrt(r2);
                }
                ++c;
            }
            if (!pass) cnt[i] = c;
        }
        if (!pass) { /* exclusive prefix over i */
            int64_t run = 0;
            for (int64_t i = 0; i < n; ++i) {
                int64_t c = cnt[i];
                cnt[i] = run;
                run += c;
            }
            cnt[n] = run;
        }
    }
    *npairs = cnt[n];
    free(cnt);
    return 0;
}

/* The cut-off radius of every type pair (ntypes x ntypes into rc_out): the rcut
 * table, except WCA's 2^(1/6) sigma.  Returns -1 on a missing table. */
int oracle_cutoffs(int32_t ntypes, int32_t kind, const double *eps, const double *sigma,
                   const double *rcut, const double *pa, const double *pb, double *rc_out)
{
    pair_model m;
    if (ntypes < 1 || !rc_out || make_model(&m, ntypes, kind, eps, sigma, rcut, pa, pb))
        return -1;
    resolved_cuts(&m, rc_out);
    return 0;
}

/* wrap one coordinate into [-L/2, L/2) and count the box crossings (paper silent) */
static void wrap1(double *x, int32_t *img, double L)
{
    double k = floor((*x + 0.5 * L) / L);
    *x -= k * L;
    if (*x >= 0.5 * L) {
        *x -= L;
        k += 1;
    } else if (*x < -0.5 * L) {
        *x += L;
        k -= 1;
    }
    *img += (int32_t)k;
}

void oracle_wrap(int64_t n, const double *box, double *pos, int32_t *image)
{
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) wrap1(&pos[3 * i + a], &image[3 * i + a], box[a]);
}

/* K = 1/2 m sum v^2, summed in ascending particle order */
double oracle_kinetic(int64_t n, const double *vel, double mass)
{
    double s = 0;
    for (int64_t i = 0; i < n; ++i)
        s += vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] +
             vel[3 * i + 2] * vel[3 * i + 2];
    return 0.5 * mass * s;
}

/*
 * Velocity-Verlet NVE run (Listing 1's mode_standard(dt) + run(n) with NVE in
 * place of NVT; Section 3.1 lists NVE).  pos/vel/image in and out (n x 3);
 * pos is wrapped before the first step.  force: n x 3 out, F at the final
 * positions.  Optional series (NULL to skip), each of length nsteps + 1, entry s
 * taken after step s (entry 0 = initial state): pe[s], ke[s].
 */
int oracle_vv(int64_t n, const double *box, double *pos, double *vel, int32_t *image,
              const int32_t *type, int32_t ntypes, int32_t kind, const double *eps,
              const double *sigma, const double *rcut, const double *pa, const double *pb,
              double mass, double dt, int64_t nsteps, double *force, double *pe, double *ke)
{
    pair_model m;
    if (check_common(n, box, ntypes) || nsteps < 0 || !(mass > 0) ||
        make_model(&m, ntypes, kind, eps, sigma, rcut, pa, pb))
        return -1;
    oracle_wrap(n, box, pos, image);
    double U;
    int rc = forces_model(n, box, pos, type, &m, force, &U, NULL, NULL, NULL);
    if (rc) return rc;
    if (pe) pe[0] = U;
    if (ke) ke[0] = oracle_kinetic(n, vel, mass);
    double h = 0.5 * dt / mass;
    for (int64_t s = 1; s <= nsteps; ++s) {
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] += h * force[i];
        for (int64_t i = 0; i < 3 * n; ++i) pos[i] += dt * vel[i];
        oracle_wrap(n, box, pos, image);
        rc = forces_model(n, box, pos, type, &m, force, &U, NULL, NULL, NULL);
        if (rc) return rc;
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] += h * force[i];
        if (pe) pe[s] = U;
        if (ke) ke[s] = oracle_kinetic(n, vel, mass);
    }
    return 0;
}

/* NVT with a Nose-Hoover thermostat in the Martyna-Tobias-Klein form (Section 3.1:
 * the NVT, NPH and NPT integrators follow Martyna, Tobias and Klein; Listing 1 uses
 * NVT with kT and tau).  The paper prints no equation; the textbook equations are
 *   dx/dt = v,  dv/dt = F/m - xi v,  dxi/dt = (2K/(g kT) - 1) / tau^2,  deta/dt = xi
 * with g = 3N - 3 degrees of freedom (the temperature convention used here), and
 *   H = K + U + g kT (tau^2 xi^2 / 2 + eta)
 * is conserved.  One step of the time-reversible splitting:
 *   xi += dt/2 G(K);  v *= exp(-xi dt/2);  eta += dt/2 xi;
 *   v += dt/(2m) F;  x += dt v;  wrap;  F = F(x);  v += dt/(2m) F;
 *   v *= exp(-xi dt/2);  eta += dt/2 xi;  xi += dt/2 G(K)
 * with G(K) = (2K/(g kT) - 1)/tau^2 and K from the velocities of that moment.
 * xi_io / eta_io hold the thermostat on entry and on return; the optional series
 * (nsteps + 1 entries) record U, K, xi, eta after each step (entry 0: the start). */
int oracle_nvt(int64_t n, const double *box, double *pos, double *vel, int32_t *image,
               const int32_t *type, int32_t ntypes, int32_t kind, const double *eps,
               const double *sigma, const double *rcut, const double *pa, const double *pb,
               double mass, double dt, double kT, double tau, int64_t nsteps, double *force,
               double *xi_io, double *eta_io, double *pe, double *ke, double *xis,
               double *etas)
{
    pair_model m;
    if (check_common(n, box, ntypes) || nsteps < 0 || !(mass > 0) || !(kT > 0) || !(tau > 0) ||
        n < 2 || !xi_io || !eta_io || make_model(&m, ntypes, kind, eps, sigma, rcut, pa, pb))
        return -1;
    const double g = 3.0 * (double)n - 3.0;
    double xi = *xi_io, eta = *eta_io;
    oracle_wrap(n, box, pos, image);
    double U;
    int rc = forces_model(n, box, pos, type, &m, force, &U, NULL, NULL, NULL);
    if (rc) return rc;
    if (pe) pe[0] = U;
    if (ke) ke[0] = oracle_kinetic(n, vel, mass);
    if (xis) xis[0] = xi;
    if (etas) etas[0] = eta;
    const double h = 0.5 * dt / mass;
    for (int64_t s = 1; s <= nsteps; ++s) {
        double K = oracle_kinetic(n, vel, mass);
        xi += 0.5 * dt * (2.0 * K / (g * kT) - 1.0) / (tau * tau);
        double sc = exp(-0.5 * dt * xi);
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] *= sc;
        eta += 0.5 * dt * xi;
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] += h * force[i];
        for (int64_t i = 0; i < 3 * n; ++i) pos[i] += dt * vel[i];
        oracle_wrap(n, box, pos, image);
        rc = forces_model(n, box, pos, type, &m, force, &U, NULL, NULL, NULL);
        if (rc) return rc;
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] += h * force[i];
        sc = exp(-0.5 * dt * xi);
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] *= sc;
        eta += 0.5 * dt * xi;
        K = oracle_kinetic(n, vel, mass);
        xi += 0.5 * dt * (2.0 * K / (g * kT) - 1.0) / (tau * tau);
        if (pe) pe[s] = U;
        if (ke) ke[s] = K;
        if (xis) xis[s] = xi;
        if (etas) etas[s] = eta;
    }
    *xi_io = xi;
    *eta_io = eta;
    return 0;
}

/* T = 2K/(3N-3) and P = (N T + tr(W)/3) / V from K and the virial (paper silent) */
void oracle_thermo(int64_t n, const double *box, double ke, const double *virial, double *T,
                   double *P)
{
    double dof = 3.0 * (double)n - 3.0;
    double t = dof > 0 ? 2.0 * ke / dof : 0.0;
    double vol = box[0] * box[1] * box[2];
    double trw = virial[0] + virial[3] + virial[5];
    *T = t;
    *P = ((double)n * t + trw / 3.0) / vol;
}
