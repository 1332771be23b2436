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

/* All interactions of particle i (j runs over every other particle, ascending).
 * Outputs the force on i, half of its pair energies and half of its pair virials. */
static void particle_terms(int64_t i, int64_t n, const double *box, const double *pos,
                           const int32_t *type, int32_t ntypes, const double *eps,
                           const double *sigma, const double *rcut, double f_out[3],
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
        int32_t p = ti * ntypes + type[j];
        double rc = rcut[p];
        if (!(r2 < rc * rc)) continue;
        double v, f;
        lj_pair(r2, eps[p], sigma[p], rc, &v, &f);
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

/*
 * Forces, total potential energy and virial tensor of the whole system.
 * pos: n x 3 row-major, any image.  eps/sigma/rcut: ntypes x ntypes row-major.
 * force: n x 3 out.  energy: scalar out.  virial: 6 out (xx,xy,xz,yy,yz,zz).
 * per_energy / per_virial: optional (NULL) per-particle halves (n, n x 6).
 */
int oracle_forces(int64_t n, const double *box, const double *pos, const int32_t *type,
                  int32_t ntypes, const double *eps, const double *sigma, const double *rcut,
                  double *force, double *energy, double *virial, double *per_energy,
                  double *per_virial)
{
    if (check_common(n, box, ntypes)) return -1;
    double *u = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *w = (double *)malloc(sizeof(double) * 6 * (size_t)(n > 0 ? n : 1));
    if (!u || !w) {
        free(u);
        free(w);
        return -2;
    }
#pragma omp parallel for schedule(dynamic, 16) num_threads(oracle_get_threads())
    for (int64_t i = 0; i < n; ++i)
        particle_terms(i, n, box, pos, type, ntypes, eps, sigma, rcut, &force[3 * i], &u[i],
                       &w[6 * i]);
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
                         int32_t ntypes, const double *eps, const double *sigma,
                         const double *rcut, int64_t m, const int64_t *idx, double *force,
                         double *per_energy, double *per_virial)
{
    if (check_common(n, box, ntypes) || m < 0) return -1;
    for (int64_t k = 0; k < m; ++k)
        if (idx[k] < 0 || idx[k] >= n) return -1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(oracle_get_threads())
    for (int64_t k = 0; k < m; ++k) {
        double u, w[6];
        particle_terms(idx[k], n, box, pos, type, ntypes, eps, sigma, rcut, &force[3 * k], &u,
                       w);
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
              const int32_t *type, int32_t ntypes, const double *eps, const double *sigma,
              const double *rcut, double mass, double dt, int64_t nsteps, double *force,
              double *pe, double *ke)
{
    if (check_common(n, box, ntypes) || nsteps < 0 || !(mass > 0)) return -1;
    oracle_wrap(n, box, pos, image);
    double U;
    int rc = oracle_forces(n, box, pos, type, ntypes, eps, sigma, rcut, force, &U, NULL, NULL,
                           NULL);
    if (rc) return rc;
    if (pe) pe[0] = U;
    if (ke) ke[0] = oracle_kinetic(n, vel, mass);
    double h = 0.5 * dt / mass;
    for (int64_t s = 1; s <= nsteps; ++s) {
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] += h * force[i];
        for (int64_t i = 0; i < 3 * n; ++i) pos[i] += dt * vel[i];
        oracle_wrap(n, box, pos, image);
        rc = oracle_forces(n, box, pos, type, ntypes, eps, sigma, rcut, force, &U, NULL, NULL,
                           NULL);
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
               const int32_t *type, int32_t ntypes, const double *eps, const double *sigma,
               const double *rcut, double mass, double dt, double kT, double tau,
               int64_t nsteps, double *force, double *xi_io, double *eta_io, double *pe,
               double *ke, double *xis, double *etas)
{
    if (check_common(n, box, ntypes) || nsteps < 0 || !(mass > 0) || !(kT > 0) || !(tau > 0) ||
        n < 2 || !xi_io || !eta_io)
        return -1;
    const double g = 3.0 * (double)n - 3.0;
    double xi = *xi_io, eta = *eta_io;
    oracle_wrap(n, box, pos, image);
    double U;
    int rc = oracle_forces(n, box, pos, type, ntypes, eps, sigma, rcut, force, &U, NULL, NULL,
                           NULL);
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
        rc = oracle_forces(n, box, pos, type, ntypes, eps, sigma, rcut, force, &U, NULL, NULL,
                           NULL);
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
