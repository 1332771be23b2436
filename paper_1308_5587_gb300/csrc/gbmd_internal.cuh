// gbmd_internal.cuh -- device-side data layout shared by the kernels of libgbmd.
//
// Every kernel walks a tile table (system, first, count) over a device array of
// SysDev descriptors, so one launch serves one system or a whole batch, and the
// descriptors (not the launch arguments) hold buffer pointers and sizes: a
// captured CUDA graph stays valid when a buffer is re-allocated (neighbour-list
// growth) because only the descriptor in device memory changes.
//
// Data layout per system (N particles, current internal order):
//   x, v        FP64 planar [3][N] (x wrapped into [-L/2, L/2); v lags half a kick
//               behind the full-step velocity unless flags->v_full)
//   img         int32 planar [3][N] periodic image counts
//   type, tag   int32 [N]; rtag int32 [N] (tag -> internal index)
//   q           int4 [N]: x as 32-bit fixed point of x/L (2^32 <-> L, two's
//               complement, so an int32 difference is the minimum image) + type in w
//   q_build     int4 [N]: q at the last neighbour-list build (displacement check)
//   p64         double4_32a [N]: FP64 x, y, z + type bits in w (FP64 force gather only)
//   f32 / f64   float4 / double4_32a [N]: force (+ per-particle energy in w when asked)
//   nn, nl      int32 [N] neighbour counts; ELL4 list: entry k of particle i at
//               nl[((k / 4) * nl_stride + i) * 4 + k % 4], nl_stride = N rounded up
//               to 32, cap (a multiple of 4) entries per particle
//   cell arrays key [N] (cell rank), cnt/start/cursor [ncells+1], members [N]
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gbmd.h"
#include "tree_core.cuh"

namespace gbmd {

constexpr int MAXT = GBMD_MAX_TYPES;
constexpr int MAXT2 = MAXT * MAXT;

// error codes stored in Flags::error (positive on the device)
enum DevError : int { DEV_OK = 0, DEV_OVERFLOW = 1, DEV_NONFINITE = 2, DEV_BADTYPE = 3, DEV_WINDOW = 4,
                      DEV_TREE = 5 /* a tree traversal ran past its node bound */ };

// staged force tiles: aligned 2x2x2 blocks of cells; their 4x4x4-cell window is
// staged in shared memory (at most window_cap particles)
constexpr int WIN_CELLS = 64;

struct Flags {
  int rebuild_req;          // set by the step kernel when r_buff/2 is exceeded
  int do_rebuild;           // this step rebuilds (decided once per step)
  int do_sort;              // this step re-sorts (Morton cell order) before building
  int active;               // this step advances the system
  int error;                // DevError; nonzero freezes the system
  int overflow_need;        // largest neighbour count seen in an overflowing build
  int v_full;               // 1: v holds full-step velocities (after create / set_state)
  int max_window;           // largest staged window of the last build (particles)
  long long step;           // steps completed
  long long step_limit;     // -1 = none
  long long last_sort;      // step of the last Morton re-sort
  long long n_rebuilds;
  long long n_sorts;
  unsigned long long launches;   // kernels executed for this system
  unsigned long long nb_total;   // sum of neighbour counts at the last build
};

static_assert(sizeof(Flags) == 88 && offsetof(Flags, step) == 32, "Flags layout");

// Device reads of a system's flags, which other blocks and kernels of the step
// write: volatile vector loads, so that the fields a kernel needs arrive in one
// round trip instead of one dependent load each.  Flags sit at the start of their
// own cudaMalloc allocation (256-byte aligned).
struct FlagWords {
  int rebuild_req, do_rebuild, do_sort, active;   // bytes 0..15
  int error, overflow_need, v_full, max_window;   // bytes 16..31
};
__device__ __forceinline__ FlagWords load_flag_words(const Flags* f) {
  FlagWords w;
  asm volatile("ld.volatile.global.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(w.rebuild_req), "=r"(w.do_rebuild), "=r"(w.do_sort), "=r"(w.active)
               : "l"(f));
  asm volatile("ld.volatile.global.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(w.error), "=r"(w.overflow_need), "=r"(w.v_full), "=r"(w.max_window)
               : "l"(reinterpret_cast<const char*>(f) + 16));
  return w;
}
// (step, step_limit) and (last_sort, n_rebuilds)
__device__ __forceinline__ longlong2 load_flag_pair(const long long* p) {
  longlong2 r;
  asm volatile("ld.volatile.global.v2.s64 {%0, %1}, [%2];" : "=l"(r.x), "=l"(r.y) : "l"(p));
  return r;
}

// Per type-pair coefficients of the pair evaluators (k_force.cuh); rc2 = r_cut^2,
// rl2 = (r_cut + r_buff)^2, shift = the unshifted V(r_cut).  p0..p4 by evaluator:
//   LJ (and WCA):  p0 = 48 eps sigma^12, p1 = 24 eps sigma^6 (force factors),
//                  p3 = 4 eps sigma^12, p4 = 4 eps sigma^6 (energy)
//   Mie:           p0 = sigma^2, p1 = n/2, p2 = m/2, p3 = C eps
//   Yukawa:        p0 = eps, p1 = kappa
//   Gaussian:      p0 = eps, p1 = 1/(2 sigma^2), p2 = eps/sigma^2
// (unused entries are 0)
struct PairF { float p0, p1, rc2, p2; float p3, p4, shift, rl2; };
struct PairD { double p0, p1, rc2, rl2; double p3, p4, shift, p2; };

// the pair evaluators of the force kernels (WCA runs the LJ one)
enum PairEval : int { EVAL_LJ = GBMD_POT_LJ, EVAL_MIE = GBMD_POT_MIE,
                      EVAL_YUKAWA = GBMD_POT_YUKAWA, EVAL_GAUSS = GBMD_POT_GAUSS };
inline int eval_of(int potential) {
  return potential == GBMD_POT_WCA ? EVAL_LJ : potential;
}

struct SysDev {
  // geometry
  double L[3], halfL[3];
  double qscale[3];        // 2^32 / L
  float fscale[3];         // L / 2^32
  float rbuff_half2;       // (r_buff / 2)^2, slightly reduced (conservative)
  int nc[3];               // cells per axis
  int ncells;
  // sort bins of the cell list: ncells, or ntypes * ncells (type-major: bin =
  // type * ncells + cell rank) for the tree neighbour list
  int nbins;
  // tree neighbour list (k_tree.cu; tree_core.cuh): after each sort, type t's
  // particles are members[tree_first[t] .. + tree_n[t]); its tree has tree_P[t]
  // leaves (global leaf numbers tree_leaf0[t] ..) and boxes
  // tree_box[tree_node0[t] + 1 .. + 2 tree_P[t] - 1]
  int tree;
  int tree_first[MAXT], tree_n[MAXT], tree_P[MAXT], tree_leaf0[MAXT], tree_node0[MAXT];
  int tree_leaves_total;
  TreeBox* tree_box;
  unsigned* tree_arrive;   // per node: children arrived during the build (reset to 0)
  unsigned* fkey;          // [N] the particle's fine Morton code at the last build (every
                           // system: the order inside a cell)
  int4* cpos;              // [N] position shadow of member m (cell order) at the last build
  int4* tree_q;            // [N] the leaves' particles in leaf order: (x, y, z, index)
  // the list kernel visits the types in decreasing order of their expected query work
  // (sum over t of n_t r_list(type, t)^3): launch positions tree_qpos[k] .. belong to
  // type tree_qtype[k]
  int tree_qpos[MAXT + 1], tree_qtype[MAXT];
  int n, ntypes, cap, precision;
  // domain decomposition: the last n_ghost tags are ghosts (not integrated; their
  // positions are set from outside every step); such a system leaves its rebuilds to
  // the caller (the step records rebuild_req and does not act on it)
  int n_ghost;
  int nl_stride;           // particles per slot group of the list (N rounded up to 32)
  // staged force path (mixed precision, >= 4 cells per axis): the list holds 16-bit
  // window-local indices in ELL8 layout, indexed by member rank (cell order)
  int staged;
  int nb[3], nblocks;      // 2x2x2 cell blocks per axis, total
  int window_cap;          // window particles that fit the staged kernel's shared memory
  int2 *blk_win;           // [nblocks][64]: (member start, window offset) per window cell
  int4 *blk_info;          // [nblocks]: (first member, particles, window total, 0)
  int *rmember;            // particle index -> member rank
  int sort_period;
  double dt, h;            // h = dt / (2 m)
  // NVT (Nose-Hoover, MTK form): nh = {xi, eta, exp(-xi dt/2), 0} on the device;
  // nh_part: the group's per-step-tile partial sums of v.v; tile_first_s /
  // tile_count_s: this system's tiles of the step's force launch
  int nvt;
  double kT, tau, gdof;    // gdof = 3N - 3
  double* nh;
  double* nh_part;
  int tile_first_s, tile_count_s;
  double dtq[3];           // dt * 2^32 / L: the drift in box-fraction units
  double mass;
  int eval;                // PairEval of the system's potential
  // per type pair
  PairF pf[MAXT2];
  PairD pd[MAXT2];
  // particle arrays
  double *x, *v;
  int *img, *type, *tag, *rtag;
  // position shadows, double-buffered by step parity (q, p64: even steps; q1, p64b:
  // odd steps): the step kernel gathers from one and writes the next step's to the
  // other.  p64 only in FP64 mode.
  int4 *q, *q1, *q_build;
  double4_32a *p64, *p64b;
  float4 *f32;
  double4_32a *f64;
  int *nn, *nl;
  // cell list
  int *key, *cell_cnt, *cell_start, *cell_cursor, *members, *members_tmp;
  const int *rank2lin, *lin2rank;
  // re-sort scratch (same layout as the primaries)
  double *x_alt, *v_alt;
  int *img_alt, *type_alt, *tag_alt;
  int4 *q_alt;
  // thermo scratch: per-force-tile partial sums (pe, virial[6], pad) and output
  double *partials;
  int tile_first_f, tile_count_f;   // this system's tiles in the force tile table
  double *thermo;                   // 16 doubles: pe, ke, virial[6], ...
  double *pp_u, *pp_w;              // optional per-particle energy / virial (N, N x 6)
  Flags *flags;
};

// group-level control block (one per single system or batch)
struct GroupCtl {
  unsigned int blocks_done;  // last-block counter of the step kernel
  unsigned int blocks_done_a;   // last-block counter of the NVT force half
  int any_rebuild;
  unsigned long long launches;
};

struct Tile { int sys, first, count, pad; };

// ---- device helpers -------------------------------------------------------

// a system's step counter (written by the last block of each step)
__device__ __forceinline__ long long step_of(const Flags* f) {
  long long r;
  asm volatile("ld.volatile.global.s64 %0, [%1];" : "=l"(r) : "l"(&f->step));
  return r;
}
// the shadow of the positions at step `step` (and the buffer for step + 1)
__device__ __forceinline__ int4* q_at(const SysDev& s, long long step) {
  return (step & 1) ? s.q1 : s.q;
}
__device__ __forceinline__ double4_32a* p64_at(const SysDev& s, long long step) {
  return (step & 1) ? s.p64b : s.p64;
}

__device__ __forceinline__ void count_launch(const SysDev& s) {
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&s.flags->launches, 1ull);
}

// 32-bit fixed point of x/L with wrap-around; x in any image
__device__ __forceinline__ int to_fixed(double x, double qscale) {
  long long q = __double2ll_rn(x * qscale);
  return (int)(unsigned int)(unsigned long long)q;
}

__device__ __forceinline__ int min_image_fixed(int a, int b) {
  return (int)((unsigned int)a - (unsigned int)b);
}

// address of entry k of particle i in the ELL4 neighbour list
__device__ __forceinline__ size_t nl_index(int i, int k, int stride) {
  return ((size_t)(k >> 2) * (size_t)stride + (size_t)i) * 4 + (size_t)(k & 3);
}

// address of entry k of member m in the staged (ELL8, 16-bit) neighbour list
__device__ __forceinline__ size_t nl16_index(int m, int k, int stride) {
  return ((size_t)(k >> 3) * (size_t)stride + (size_t)m) * 8 + (size_t)(k & 7);
}

// cell coordinate of a fixed-point coordinate: floor((q + 2^31) * nc / 2^32)
__device__ __forceinline__ int cell_of_fixed(int q, int nc) {
  unsigned long long u = (unsigned long long)((unsigned int)q ^ 0x80000000u);
  return (int)((u * (unsigned long long)nc) >> 32);
}

}  // namespace gbmd
