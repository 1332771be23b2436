/*
 * gbmd.h -- C ABI of libgbmd, a GB300 (sm_103a) Lennard-Jones molecular-dynamics
 * hot path: cell list, Verlet neighbour list with skin, LJ pair force and a fused
 * velocity-Verlet NVE step, for one system or for many systems stepped together.
 * The same gather also evaluates the other short-range pair potentials Section 3.1
 * lists beside LJ (Mie, WCA, Yukawa, Gaussian; gbmd_desc.potential).
 *
 * The calls follow the HOOMD-blue paper's statement of the problem:
 *   - a system is particles with positions and types in a periodic box
 *     (Section 3.1, Listing 1: init.create_lattice);
 *   - forces come from md.pair.lj(r_cut) with per type-pair epsilon and sigma
 *     (Listing 1, pair_coeff.set), gathered from a cell-based neighbour list
 *     (md.nlist.cell);
 *   - md.integrate.mode_standard(dt) advances it; run(n) steps it n times
 *     (Listing 1; NVE is among the ensembles of Section 3.1);
 *   - results are force, energy and virial (Section 7.1).
 * The paper gives no equations; the library computes:
 *   V(r) = 4 eps[(sigma/r)^12 - (sigma/r)^6] - V_LJ(r_cut) for r < r_cut, else 0;
 *   F_ij = 24 eps [2 (sigma/r)^12 - (sigma/r)^6] / r^2 * d_ij, d_ij = x_i - x_j
 *   (minimum image); U = sum_{i<j} V; W_ab = sum_{i<j} d_ij,a F_ij,b;
 *   K = 1/2 m sum v^2; T = 2K/(3N-3); P = (N T + tr W / 3) / V;
 *   velocity Verlet: v += dt/(2m) F; x += dt v; wrap; F = F(x); v += dt/(2m) F.
 * The neighbour list holds every pair with r < r_cut,ij + r_buff at its last
 * build and is rebuilt when some particle has moved more than r_buff/2 since.
 *
 * Conventions for every call:
 *   - Host arrays are row-major N x 3 (x, y, z per particle) in TAG order, the
 *     order of the arrays given at creation; the library may reorder particles
 *     internally (Morton/cell order) but every output is in tag order.
 *   - The caller keeps ownership of every array it passes; the library copies
 *     what it needs.  Output arrays are caller-allocated.
 *   - Positions may be given in any periodic image; the library wraps them into
 *     the centred box [-L/2, L/2) and keeps integer image counts.
 *   - Return value: GBMD_OK (0) or a negative gbmd_status.  The library never
 *     aborts the process and never traps on the device; device-side faults
 *     (neighbour-list overflow, non-finite coordinates) are recorded in device
 *     memory and reported by the next call that synchronises.  On error,
 *     gbmd_last_error() returns a message for the calling thread.
 *   - Asynchrony: gbmd_step / gbmd_batch_step only enqueue work on the system's
 *     CUDA stream.  Every gbmd_get_* call synchronises that stream first.
 */
#ifndef GBMD_H
#define GBMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBMD_ABI_VERSION 6
#define GBMD_MAX_TYPES 4

typedef enum gbmd_status {
    GBMD_OK = 0,
    GBMD_ERR_BAD_ARG = -1,          /* invalid argument (null pointer, size, parameter) */
    GBMD_ERR_BOX_TOO_SMALL = -2,    /* some box edge < 2 (r_cut,max + r_buff) */
    GBMD_ERR_OOM = -3,              /* device allocation failed */
    GBMD_ERR_NLIST_OVERFLOW = -4,   /* neighbour list overflow that could not be recovered */
    GBMD_ERR_NONFINITE = -5,        /* a coordinate became NaN/Inf, or moved > L/2 in a step */
    GBMD_ERR_CUDA = -6,             /* a CUDA runtime call failed */
    GBMD_ERR_TIMEOUT = -7,          /* a bounded wait ran out */
    GBMD_ERR_STATE = -8,            /* call not valid in the current state (e.g. in a batch) */
    GBMD_ERR_NO_DEVICE = -9         /* no usable CUDA device */
} gbmd_status;

typedef enum gbmd_precision {
    GBMD_FP64 = 0,   /* every step in FP64 */
    GBMD_MIXED = 1   /* FP32 pair forces and sums; FP64 positions, wrap, integration, reductions */
} gbmd_precision;

/* System description.  All pointers are read during gbmd_create* only. */
typedef struct gbmd_desc {
    int64_t n;                  /* number of particles, >= 1 */
    double box[3];              /* orthorhombic box edges Lx, Ly, Lz (> 0) */
    const double *pos;          /* n x 3 positions (any image) */
    const double *vel;          /* n x 3 velocities */
    const int32_t *type;        /* n type ids in [0, ntypes); NULL = all type 0 */
    const int32_t *image;       /* n x 3 initial image counts; NULL = all 0 */
    int32_t ntypes;             /* 1 .. GBMD_MAX_TYPES */
    const double *eps;          /* ntypes x ntypes, symmetric, > 0 (finite, nonzero for
                                   Yukawa and Gaussian) */
    const double *sigma;        /* ntypes x ntypes, symmetric, > 0 (unread for Yukawa) */
    const double *rcut;         /* ntypes x ntypes, symmetric, > 0 (r_cut per pair; unread
                                   for WCA) */
    double r_buff;              /* neighbour-list skin, >= 0 */
    double dt;                  /* time step, > 0 */
    double mass;                /* particle mass, > 0 */
    int32_t precision;          /* gbmd_precision */
    int32_t sort_period;        /* re-sort particles into Morton cell order at the first
                                   rebuild at least this many steps after the last sort;
                                   0 = sort only when the system is created */
    int32_t nlist_capacity;     /* neighbours per particle to reserve; 0 = from density */
    int32_t threads_per_particle; /* lanes per particle in the force kernel:
                                     0 = default (1 from 2^19 particles up, else 2);
                                     else 1, 2 or 4 */
    void *stream;               /* cudaStream_t to run on; NULL = the legacy default stream */
    int32_t device;             /* CUDA device ordinal; -1 = the calling thread's current
                                   device.  Every later call on the system uses it. */
    int32_t force_path;         /* GBMD_PATH_GLOBAL (0, default): the force kernel gathers
                                   neighbour positions through L1/L2 by 32-bit index.
                                   GBMD_PATH_STAGED (1): mixed precision only; each block
                                   of 2x2x2 cells stages its 4x4x4-cell window in shared
                                   memory and the list holds 16-bit window indices.  Used
                                   only where every cell axis has >= 4 cells and the
                                   expected window fits; a window that outgrows shared
                                   memory at a rebuild switches the system to the global
                                   path for good.  gbmd_get_info reports the path in use. */
    int32_t integrator;         /* GBMD_NVE (0): velocity Verlet.  GBMD_NVT (1): Nose-Hoover
                                   thermostat in the Martyna-Tobias-Klein form (Section 3.1;
                                   Listing 1's md.integrate.nvt(kT, tau)): dv/dt = F/m - xi v,
                                   dxi/dt = (2K/(g kT) - 1)/tau^2, g = 3N - 3, integrated by
                                   the time-reversible splitting xi/2, scale/2, velocity
                                   Verlet, scale/2, xi/2.  NVT uses the global force path. */
    double kT;                  /* NVT target temperature (> 0) */
    double tau;                 /* NVT coupling time (> 0) */
    int32_t potential;          /* the pair potential (gbmd_potential; 0 = LJ).  Every one
                                   is truncated at r_cut,ij and shifted by its value there
                                   (the force is not shifted), d_ij = x_i - x_j,
                                   F_ij = f(r) d_ij:
                                   GBMD_POT_LJ: the 12-6 form above.
                                   GBMD_POT_MIE: V = C eps [(sigma/r)^n - (sigma/r)^m],
                                     C = n/(n-m) (n/m)^(m/(n-m)) (depth -eps at the
                                     minimum), f = C eps [n (sigma/r)^n - m (sigma/r)^m]/r^2;
                                     n, m from mie_n, mie_m (n > m > 0, real).
                                   GBMD_POT_WCA: the 12-6 form cut at its minimum:
                                     r_cut,ij = 2^(1/6) sigma_ij; rcut is not read (may be
                                     NULL); V = 4 eps [...] + eps >= 0.
                                   GBMD_POT_YUKAWA: V = eps exp(-kappa r)/r,
                                     f = eps exp(-kappa r) (1 + kappa r)/r^3; kappa >= 0
                                     from `kappa`; sigma is not read (may be NULL); eps may
                                     have either sign.
                                   GBMD_POT_GAUSS: V = eps exp(-r^2/(2 sigma^2)),
                                     f = eps/sigma^2 exp(-r^2/(2 sigma^2)); eps may have
                                     either sign.
                                   Systems stepped together in one batch share the
                                   evaluator (LJ and WCA share one).  The staged force path
                                   serves LJ and WCA only; the others use the global one. */
    const double *mie_n;        /* ntypes x ntypes, symmetric (GBMD_POT_MIE; else unread) */
    const double *mie_m;        /* ntypes x ntypes, symmetric, 0 < m < n (GBMD_POT_MIE) */
    const double *kappa;        /* ntypes x ntypes, symmetric, >= 0 (GBMD_POT_YUKAWA) */
    int32_t nlist;              /* how the neighbour list is built (the list itself, every
                                   pair with r < r_cut,ij + r_buff, is the same):
                                   GBMD_NLIST_CELL (0, default): cell list of width
                                   >= r_list,max, 27-cell stencil (Listing 1's
                                   md.nlist.cell).
                                   GBMD_NLIST_TREE (1): a bounding volume hierarchy per
                                   particle type, each particle querying every type's
                                   tree with its own r_list,ij (Section 5: nlist.tree,
                                   for size-disperse systems, where cells sized to the
                                   largest particles hold many small ones).  Uses the
                                   global force path. */
    int64_t n_ghost;            /* Ghost particles, for a system that is one domain of a
                                   spatially decomposed one (the paper's MPI domain
                                   decomposition, Sections 2 and 5): the last n_ghost
                                   particles in tag order are copies of particles owned by
                                   other domains (the halo).  They exert forces on the
                                   others but are not integrated: their positions are
                                   replaced by gbmd_set_ghost_positions before every step,
                                   and their own forces, velocities and energies mean
                                   nothing.  Such a system does not rebuild its lists by
                                   itself: once one of its own particles has moved more
                                   than r_buff/2 since the last build, gbmd_get_info
                                   reports rebuild_pending and the caller rebuilds every
                                   domain (re-partitioning and recreating them, or
                                   gbmd_set_state).  0 <= n_ghost < n; ghosts need the NVE
                                   integrator and the global force path, and a system with
                                   ghosts cannot join a batch.  Readouts cover every
                                   particle, ghosts included.  0 = none. */
} gbmd_desc;

enum { GBMD_PATH_GLOBAL = 0, GBMD_PATH_STAGED = 1 };
enum { GBMD_NVE = 0, GBMD_NVT = 1 };
enum { GBMD_NLIST_CELL = 0, GBMD_NLIST_TREE = 1 };
typedef enum gbmd_potential {
    GBMD_POT_LJ = 0,
    GBMD_POT_MIE = 1,
    GBMD_POT_WCA = 2,
    GBMD_POT_YUKAWA = 3,
    GBMD_POT_GAUSS = 4
} gbmd_potential;

/* Thermodynamic quantities of one system at its current step (FP64). */
typedef struct gbmd_thermo {
    int64_t step;
    double pe;          /* U = sum_{i<j} V(r_ij) */
    double ke;          /* K = 1/2 m sum v^2 at full-step velocities */
    double temperature; /* 2K / (3N - 3) */
    double pressure;    /* (N T + tr W / 3) / V */
    double virial[6];   /* W: xx, xy, xz, yy, yz, zz */
    double w;           /* tr W */
    int64_t n_rebuilds; /* neighbour-list builds since creation */
    double xi;          /* NVT thermostat variable (0 for NVE) */
    double eta;         /* NVT thermostat position, d eta / dt = xi (0 for NVE) */
    double h_ext;       /* conserved quantity: K + U, plus g kT (tau^2 xi^2 / 2 + eta) for NVT */
} gbmd_thermo;

/* Configuration and counters of one system, for diagnostics and benchmarks. */
typedef struct gbmd_info {
    int64_t n;
    int32_t precision;
    int32_t ntypes;
    int32_t cells[3];             /* cells per axis of the cell list */
    int32_t nlist_capacity;       /* current neighbours-per-particle capacity */
    int32_t threads_per_particle; /* lanes cooperating on one particle in the force kernel */
    int32_t force_block;          /* threads per block of the force kernel */
    int64_t step;
    int64_t n_rebuilds;
    int64_t n_sorts;
    int64_t kernel_launches;      /* kernels of this library executed for this system
                                     (counted on the device) */
    int64_t neighbors_total;      /* sum of neighbour counts at the last build */
    int64_t footprint_bytes;      /* device memory held */
    int32_t force_path;           /* 0: global neighbour indices; 1: staged windows (2x2x2
                                     cell blocks with their 4x4x4-cell neighbourhood in
                                     shared memory, 16-bit window-local indices) */
    int32_t max_window;           /* largest staged window at the last build (particles) */
    double cell_scale;            /* cells are at least cell_scale * r_list,max wide (tree
                                     list: r_list,min; its cells only order the particles) */
    int32_t nlist;                /* GBMD_NLIST_CELL or GBMD_NLIST_TREE */
    int32_t rebuild_pending;      /* systems with ghosts: one of the system's own
                                     particles has moved more than r_buff/2 since the last
                                     build, so every domain must be rebuilt before the
                                     next step (always 0 without ghosts, which rebuild by
                                     themselves) */
    int64_t n_ghost;              /* ghost particles (gbmd_desc.n_ghost) */
} gbmd_info;

typedef struct gbmd_system gbmd_system;
typedef struct gbmd_batch gbmd_batch;

/* ---- single system ---------------------------------------------------------- */

/* Create a system from HOST arrays: uploads, wraps, builds the cell and
 * neighbour lists and computes the initial forces.  *out receives the handle.
 * Errors: BAD_ARG, BOX_TOO_SMALL, OOM, CUDA, NO_DEVICE. */
int gbmd_create(const gbmd_desc *d, gbmd_system **out);

/* As gbmd_create, but pos, vel, type and image are DEVICE pointers (same
 * layout, e.g. from torch tensors); the library copies them on d->stream. */
int gbmd_create_device(const gbmd_desc *d, gbmd_system **out);

/* Free every device and host resource of the system (synchronises). */
int gbmd_destroy(gbmd_system *s);

/* Enqueue nsteps velocity-Verlet steps (Listing 1's run(n)) on the system's
 * stream and return without waiting.  nsteps >= 0.  Device-side errors surface
 * at the next gbmd_sync / gbmd_get_*; a neighbour-list overflow is recovered
 * there (capacity grown, the interrupted step redone, the remaining steps run).
 * STATE if the system belongs to a batch. */
int gbmd_step(gbmd_system *s, int64_t nsteps);

/* Wait for the system's queued work, recover from a neighbour-list overflow if
 * one happened, and report any other device-side error. */
int gbmd_sync(gbmd_system *s);

/* Forces on every particle at the current step, host n x 3, tag order. */
int gbmd_get_forces(gbmd_system *s, double *out);

/* Energy, virial, temperature and pressure at the current step. */
int gbmd_get_thermo(gbmd_system *s, gbmd_thermo *out);

/* Allocation-free variant of gbmd_get_thermo, for callers that must not allocate
 * GPU memory: applications whose memory manager has reserved the device's memory
 * up front (so a driver allocation would fail or fragment its pool) and code
 * that runs while another thread captures CUDA work in a mode where cudaMalloc
 * is an error.  The paper has no counterpart; it is part of this library's API
 * only.  It runs the same energy/virial kernels as gbmd_get_thermo, but their
 * per-tile partial sums and the system descriptor they read live in static
 * device arrays of this library (2 MiB + one descriptor, held on every device
 * that loads the library until the process exits) instead of in buffers the
 * library allocates.  Limits and behaviour:
 *   - systems with more than GBMD_NOALLOC_MAX_TILES energy tiles are rejected
 *     with GBMD_ERR_BAD_ARG: one tile is 128 particles on the global force path
 *     (so at most 4,194,304 particles) and one 2x2x2 block of cells on the
 *     staged path;
 *   - the first call on a device looks up the static arrays' device addresses
 *     (cudaGetSymbolAddress), once; make that first call before any stream
 *     capture begins;
 *   - it never grows buffers: if the system has a pending neighbour-list
 *     overflow or changed layout it returns GBMD_ERR_STATE (call gbmd_sync or
 *     gbmd_get_thermo once first); non-finite state gives GBMD_ERR_NONFINITE;
 *   - every call shares the static arrays, which keep the last call's contents
 *     (each call overwrites everything it reads, so nothing needs clearing);
 *     calls whose GPU work overlaps -- from two threads, or on two streams --
 *     race on them and must be serialised by the caller.
 * Output as gbmd_get_thermo (same kernels, same summation order). */
#define GBMD_NOALLOC_MAX_TILES 32768
int gbmd_get_thermo_noalloc(gbmd_system *s, gbmd_thermo *out);

/* Per-particle energy (n, half of every pair energy) and virial (n x 6, half of
 * every pair virial), tag order; either pointer may be NULL. */
int gbmd_get_per_particle(gbmd_system *s, double *energy, double *virial);

/* Checkpoint: wrapped positions, full-step velocities, image counts (n x 3 each,
 * any may be NULL) and the step counter (may be NULL). */
int gbmd_get_state(gbmd_system *s, double *pos, double *vel, int32_t *image, int64_t *step);

/* Resume: replace positions (any image), velocities and image counts (NULL image
 * = zeros) and the step counter; rebuilds the lists and recomputes forces.  Host
 * buffers, tag order, the types kept.  A non-finite position or velocity gives
 * GBMD_ERR_BAD_ARG and leaves the system as it was (checked on the device before
 * anything is replaced).  GBMD_ERR_STATE for a member of a batch. */
int gbmd_set_state(gbmd_system *s, const double *pos, const double *vel, const int32_t *image,
                   int64_t step);

/* Neighbour list of the last build, as tags: counts[n]; idx[n x cap] row-major,
 * each row sorted ascending, unused entries -1.  BAD_ARG if some particle has
 * more than cap neighbours (counts are still written). */
int gbmd_get_neighbors(gbmd_system *s, int32_t *counts, int32_t *idx, int64_t cap);

/* Configuration and counters. */
int gbmd_get_info(gbmd_system *s, gbmd_info *out);

/* Domain decomposition (Sections 2 and 5: one system split into spatial domains,
 * each on its own GPU, exchanging the positions of the particles near their
 * boundaries every step).  Replace the positions of the system's ghosts (tags
 * n - n_ghost .. n - 1): pos is n_ghost x 3 in that tag order, any periodic image,
 * in host memory (device = 0; pageable memory is copied before the call returns,
 * pinned memory must stay unchanged until the system's stream has reached the
 * copy) or device memory (device = 1).  Enqueued on the system's stream before the
 * next step, which then sees the new ghost positions.  BAD_ARG without ghosts or
 * for NULL pos; STATE while the system is in a batch. */
int gbmd_set_ghost_positions(gbmd_system *s, const double *pos, int32_t device);

/* Domain decomposition: the wrapped positions ([-L/2, L/2)) of the m particles
 * whose tags are listed (0 <= tag < n, each at most once or more), written row-major
 * m x 3 to out, after the system's queued steps.  tags and out are both host
 * memory (device = 0) or both device memory (device = 1).  Synchronises.  BAD_ARG
 * for m < 0, m > n, NULL arrays or (host tags) a tag out of range; a device tag
 * out of range gives NaN in its row. */
int gbmd_get_positions(gbmd_system *s, const int32_t *tags, int64_t m, double *out,
                       int32_t device);

/* Device bytes a system with this description would hold (for admission
 * control); returns a negative gbmd_status for an invalid description. */
int64_t gbmd_footprint_bytes(const gbmd_desc *d);

/* Stop the system from advancing once its step counter reaches `step`
 * (-1 = no limit).  Steps asked beyond the limit are skipped on the device. */
int gbmd_set_step_limit(gbmd_system *s, int64_t step);

/* Autotuner (Section 5: kernel parameters are tuned on the device at run time).
 * Chooses, by timing the candidates on this system's current state: the cell
 * width (a list rebuild at cells of 1, 1.1, 1.2 and 1.35 times r_list,max; kept
 * at 1 on the staged force path), then the force kernel's threads per particle
 * (1, 2, 4) and block size (128, 256, 512).  With a non-NULL cache_path the
 * choice is read from / appended to that text file (one line per shape: key,
 * threads per particle, block, cell scale), keyed by device, precision, type
 * mode, size and density class. */
int gbmd_autotune(gbmd_system *s, const char *cache_path);

/* Cells at least `scale` * r_list,max wide (1 <= scale <= 4; the cell list of
 * Listing 1's md.nlist.cell).  Rebuilds the cell grid, re-sorts into its Morton
 * order and rebuilds the lists and forces at the current positions; neighbour
 * sets are unchanged, the order of a particle's neighbours (and so the last bits
 * of its FP32 force) may change.  GBMD_ERR_BAD_ARG outside [1, 4]. */
int gbmd_set_cell_scale(gbmd_system *s, double scale);

/* NVT: set the thermostat variable xi and position eta, as gbmd_get_thermo
 * reports them for the state of a completed step (checkpoint/resume: after
 * gbmd_set_state, before stepping; GBMD_ERR_STATE otherwise).  GBMD_ERR_BAD_ARG for
 * an NVE system or non-finite values. */
int gbmd_set_thermostat(gbmd_system *s, double xi, double eta);

/* Set the force kernel's threads per particle (1, 2 or 4) and block size
 * (32..512, a multiple of 32) explicitly. */
int gbmd_set_tuning(gbmd_system *s, int32_t threads_per_particle, int32_t block);

/* Bracket the force kernel of every subsequent single step (gbmd_step(s, 1)) with
 * records of two CUDA events (cudaEvent_t, created by the caller with timing
 * enabled), so the caller can time that kernel inside real steps; may be called
 * between steps with new events (the step graph is updated, not rebuilt).
 * NULL, NULL removes the records.  Multi-step calls are unaffected. */
int gbmd_set_force_events(gbmd_system *s, void *ev_begin, void *ev_end);

/* ---- many systems stepped together ------------------------------------------ */

/* A batch steps all its systems with one launch per kernel per step (all systems
 * share every launch) inside captured CUDA graphs.  Every member must have the
 * batch's precision and device.  stream: cudaStream_t or NULL; device: ordinal
 * or -1 for the calling thread's current device. */
int gbmd_batch_create(int32_t precision, void *stream, int32_t device, gbmd_batch **out);

/* Add a system (between steps only).  The system's own stream is replaced by the
 * batch's while it is a member; gbmd_step on it returns STATE.  Its readouts
 * (forces, thermo, state) take the batch's force tuning from then on, also after
 * gbmd_batch_set_tuning / gbmd_batch_autotune, so that they equal those of a
 * system stepped alone at that tuning.  *slot receives a slot id for
 * gbmd_batch_remove. */
int gbmd_batch_add(gbmd_batch *b, gbmd_system *s, int32_t *slot);

/* Remove the system in `slot` (between steps; synchronises).  The system stays
 * valid and can be stepped alone or read out. */
int gbmd_batch_remove(gbmd_batch *b, int32_t slot);

/* Enqueue nsteps steps of every member (members past their step limit stay put). */
int gbmd_batch_step(gbmd_batch *b, int64_t nsteps);

/* Wait for the batch's work; recover overflowed members; report errors. */
int gbmd_batch_sync(gbmd_batch *b);

/* Autotune the batch's force kernel on its current members. */
int gbmd_batch_autotune(gbmd_batch *b, const char *cache_path);

/* Set the batch's force-kernel tuning explicitly (see gbmd_set_tuning). */
int gbmd_batch_set_tuning(gbmd_batch *b, int32_t threads_per_particle, int32_t block);

/* Number of members and total particles. */
int gbmd_batch_info(gbmd_batch *b, int32_t *members, int64_t *particles,
                    int64_t *kernel_launches);

/* Destroy the batch; members stay valid and become stand-alone again. */
int gbmd_batch_destroy(gbmd_batch *b);

/* ---- misc ------------------------------------------------------------------- */

/* Message of the last error on the calling thread ("" if none). */
const char *gbmd_last_error(void);

/* GBMD_ABI_VERSION of the loaded library. */
int gbmd_abi_version(void);

/* Arithmetic throughput probe, a measurement aid with no counterpart in the
 * paper: the denominator of the roofline of the FP64 force path, which is bound
 * by the FP64 pipe rather than by memory on this GPU (Section 5 quotes that
 * path's full-FP64 throughput on a V100).  `kind` selects the operation:
 *   GBMD_PROBE_DFMA  FP64 fused multiply-add,
 *   GBMD_PROBE_FFMA  FP32 fused multiply-add,
 *   GBMD_PROBE_DRCP  the FP64 reciprocal of the FP64 force kernel (one per pair
 *                    inside r_cut: hardware approximation plus one third-order
 *                    refinement, within 1 ulp of the correctly rounded value).
 * One launch over every SM of the current device (8 blocks of 256 threads per
 * SM, 8 independent chains per thread, `iters` >= 1 rounds) on `stream`
 * (cudaStream_t or NULL), after an untimed warm-up launch; *ops receives the
 * operations executed (a multiply-add counts as one), *ms the CUDA-event time
 * of the timed launch.  Allocates and frees a small result buffer; synchronises.
 * GBMD_ERR_BAD_ARG for an unknown kind, iters < 1 or NULL outputs. */
#define GBMD_PROBE_DFMA 0
#define GBMD_PROBE_FFMA 1
#define GBMD_PROBE_DRCP 2
int gbmd_probe_arith(int32_t kind, int32_t iters, void *stream, double *ops, float *ms);

#ifdef __cplusplus
}
#endif

#endif /* GBMD_H */
