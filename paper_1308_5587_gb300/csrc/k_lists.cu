// k_lists.cu -- cell list (integer binning + stable counting sort in Morton cell
// order), optional re-sort of the particle arrays, and the Verlet neighbour list.
//
// The paper names the structure (md.nlist.cell, Listing 1) and that HOOMD builds
// cell lists with atomic operations (Section 5); it gives no algorithm.  Here:
//   * a particle's cell comes from its 32-bit fixed-point coordinate, integer only:
//     c_a = floor((q_a + 2^31) * nc_a / 2^32), cell width L_a / nc_a >= r_list_max;
//   * cells are numbered by their rank in Morton (Z-order) of (cx, cy, cz);
//   * counting sort: atomic histogram -> exclusive scan -> atomic scatter, then
//     each cell's members are sorted by particle index, so the result is the
//     stable order (cell rank, index) whatever order the atomics ran in;
//   * neighbour list: full list (both i->j and j->i), one warp per cell whose lanes
//     are the cell's particles; every lane tests the same candidate j of the
//     neighbouring cells at a time (warp-uniform loop, broadcast loads).  Keep
//     j != i with r^2 < r_list,ij^2 (strict), r_list,ij = r_cut,ij + r_buff.  The
//     test runs in FP32 on the fixed-point difference; candidates within a relative
//     band of 1e-5 of r_list^2 are decided again in FP64 with the same operations
//     (and rounding) as the brute-force reference definition.
#include "launch.cuh"

namespace gbmd {

KernelCall make_call(void* f, int grid, int block, size_t smem);

template <typename T>
static void put(KernelCall& k, const T& v) {
  static_assert(sizeof(T) <= 16, "arg too large");
  memcpy(k.store[k.nargs], &v, sizeof(T));
  ++k.nargs;
}

__device__ __forceinline__ bool rebuilding(const SysDev& s) {
  return ((const volatile Flags*)s.flags)->do_rebuild != 0;
}
__device__ __forceinline__ bool sorting(const SysDev& s) {
  const volatile Flags* f = s.flags;
  return f->do_rebuild != 0 && f->do_sort != 0;
}
__device__ __forceinline__ void count(const SysDev& s, const Tile& t, GroupCtl* ctl) {
  if (threadIdx.x == 0 && t.first == 0) atomicAdd(&s.flags->launches, 1ull);
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
}

// ---- binning + histogram ----
__global__ void __launch_bounds__(TILE_P) k_bin(const SysDev* __restrict__ sysv,
                                                const Tile* __restrict__ tiles, GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  if (!rebuilding(s) || threadIdx.x >= t.count) return;
  const int i = t.first + threadIdx.x;
  const int4 q = s.q[i];
  const int cx = cell_of_fixed(q.x, s.nc[0]);
  const int cy = cell_of_fixed(q.y, s.nc[1]);
  const int cz = cell_of_fixed(q.z, s.nc[2]);
  const int r = s.lin2rank[(cz * s.nc[1] + cy) * s.nc[0] + cx];
  s.key[i] = r;
  atomicAdd(&s.cell_cnt[r], 1);
}

// ---- exclusive scan of the cell counts (one block per system) ----
__global__ void __launch_bounds__(SCAN_THREADS) k_scan(const SysDev* __restrict__ sysv,
                                                       const Tile* __restrict__ tiles,
                                                       GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  if (!rebuilding(s)) return;
  __shared__ int warp_tot[32];
  __shared__ int carry;
  if (threadIdx.x == 0) {
    carry = 0;
    s.flags->nb_total = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nc = s.ncells;
  for (int base = 0; base < nc; base += SCAN_THREADS) {
    const int c = base + threadIdx.x;
    const int v = c < nc ? s.cell_cnt[c] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int w = warp_tot[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_tot[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const int excl = carry + (wid ? warp_tot[wid - 1] : 0) + x - v;
    if (c < nc) {
      s.cell_start[c] = excl;
      s.cell_cursor[c] = excl;
      s.cell_cnt[c] = 0;   // ready for the next build
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) s.cell_start[nc] = carry;
}

// ---- scatter particle indices into their cells (unordered within a cell) ----
__global__ void __launch_bounds__(TILE_P) k_scatter(const SysDev* __restrict__ sysv,
                                                    const Tile* __restrict__ tiles,
                                                    GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  if (!rebuilding(s) || threadIdx.x >= t.count) return;
  const int i = t.first + threadIdx.x;
  const int p = atomicAdd(&s.cell_cursor[s.key[i]], 1);
  s.members_tmp[p] = i;
}

// ---- sort each cell's members by index (warp per cell) -> stable order ----
__global__ void __launch_bounds__(CELLS_PER_TILE * 32) k_cellsort(const SysDev* __restrict__ sysv,
                                                                  const Tile* __restrict__ tiles,
                                                                  GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!rebuilding(s) || w >= t.count) return;
  const int r = t.first + w;
  const int b = s.cell_start[r], e = s.cell_start[r + 1], n = e - b;
  if (n <= 32) {
    const int v = lane < n ? s.members_tmp[b + lane] : 0x7fffffff;
    int rk = 0;
    for (int k = 0; k < 32; ++k) rk += __shfl_sync(0xffffffffu, v, k) < v;
    if (lane < n) s.members[b + rk] = v;
  } else {
    for (int m = lane; m < n; m += 32) {
      const int v = s.members_tmp[b + m];
      int rk = 0;
      for (int k = 0; k < n; ++k) rk += s.members_tmp[b + k] < v;
      s.members[b + rk] = v;
    }
  }
}

// ---- re-sort: gather every per-particle array into cell order ----
__global__ void __launch_bounds__(TILE_P) k_permute(const SysDev* __restrict__ sysv,
                                                    const Tile* __restrict__ tiles,
                                                    GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  if (!sorting(s) || threadIdx.x >= t.count) return;
  const int k = t.first + threadIdx.x, n = s.n;
  const int o = s.members[k];
  for (int a = 0; a < 3; ++a) {
    s.x_alt[a * n + k] = s.x[a * n + o];
    s.v_alt[a * n + k] = s.v[a * n + o];
    s.img_alt[a * n + k] = s.img[a * n + o];
  }
  s.type_alt[k] = s.type[o];
  s.tag_alt[k] = s.tag[o];
  s.q_alt[k] = s.q[o];
}

__global__ void __launch_bounds__(TILE_P) k_copyback(const SysDev* __restrict__ sysv,
                                                     const Tile* __restrict__ tiles,
                                                     GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  if (!sorting(s) || threadIdx.x >= t.count) return;
  const int k = t.first + threadIdx.x, n = s.n;
  double xr[3];
  for (int a = 0; a < 3; ++a) {
    const double xq = s.x_alt[a * n + k];
    s.x[a * n + k] = xq;
    s.v[a * n + k] = s.v_alt[a * n + k];
    s.img[a * n + k] = s.img_alt[a * n + k];
    xr[a] = xq * (s.L[a] * (1.0 / 4294967296.0));
  }
  const int ty = s.type_alt[k];
  s.type[k] = ty;
  const int tg = s.tag_alt[k];
  s.tag[k] = tg;
  s.rtag[tg] = k;
  s.q[k] = s.q_alt[k];
  s.members[k] = k;
  if (s.precision == GBMD_FP64) s.p64[k] = make_double4_32a(xr[0], xr[1], xr[2], __longlong_as_double(ty));
}

// ---- FP64 decision for a candidate in the band: the reference definition ----
__device__ __noinline__ bool exact_within(const SysDev& s, int i, int j, double rl2) {
  const int n = s.n;
  double d[3];
  for (int a = 0; a < 3; ++a) {
    const double sc = s.L[a] * (1.0 / 4294967296.0);
    const double xi = __dmul_rn(s.x[a * n + i], sc);
    const double xj = __dmul_rn(s.x[a * n + j], sc);
    double dd = __dsub_rn(xi, xj);
    dd = __dsub_rn(dd, __dmul_rn(s.L[a], rint(__ddiv_rn(dd, s.L[a]))));
    d[a] = dd;
  }
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                              __dmul_rn(d[2], d[2]));
  return r2 < rl2;
}

// ---- neighbour list: one warp per cell ----
constexpr float NL_BAND = 1e-5f;

__global__ void __launch_bounds__(CELLS_PER_TILE * 32) k_nlist(const SysDev* __restrict__ sysv,
                                                               const Tile* __restrict__ tiles,
                                                               GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!rebuilding(s) || w >= t.count) return;
  const int nt = s.ntypes;
  __shared__ float rl2s[CELLS_PER_TILE][MAXT2];
  __shared__ double rl2d[CELLS_PER_TILE][MAXT2];
  for (int k = lane; k < nt * nt; k += 32) {
    rl2s[w][k] = s.pf[k].rl2;
    rl2d[w][k] = s.pd[k].rl2;
  }
  __syncwarp();
  const int r = t.first + w;
  const int nc0 = s.nc[0], nc1 = s.nc[1], nc2 = s.nc[2];
  const int lin = s.rank2lin[r];
  const int cx = lin % nc0, cy = (lin / nc0) % nc1, cz = lin / (nc0 * nc1);
  // distinct neighbour-cell offsets per axis (fewer than 3 cells: no duplicates)
  const int lo0 = nc0 >= 3 ? -1 : 0, hi0 = nc0 >= 3 ? 1 : nc0 - 1;
  const int lo1 = nc1 >= 3 ? -1 : 0, hi1 = nc1 >= 3 ? 1 : nc1 - 1;
  const int lo2 = nc2 >= 3 ? -1 : 0, hi2 = nc2 >= 3 ? 1 : nc2 - 1;
  const float fs0 = s.fscale[0], fs1 = s.fscale[1], fs2 = s.fscale[2];
  const int b = s.cell_start[r], e = s.cell_start[r + 1];
  const int cap = s.cap;
  unsigned long long nb_sum = 0;
  for (int base = b; base < e; base += 32) {
    const bool valid = base + lane < e;
    const int i = valid ? s.members[base + lane] : -1;
    const int4 qi = valid ? s.q[i] : make_int4(0, 0, 0, 0);
    const int ti = qi.w;
    int* row = s.nl + (size_t)(valid ? i : 0) * cap;
    int cnt = 0;
    for (int oz = lo2; oz <= hi2; ++oz) {
      const int z = (cz + oz + nc2) % nc2;
      for (int oy = lo1; oy <= hi1; ++oy) {
        const int y = (cy + oy + nc1) % nc1;
        for (int ox = lo0; ox <= hi0; ++ox) {
          const int x = (cx + ox + nc0) % nc0;
          const int nr = s.lin2rank[(z * nc1 + y) * nc0 + x];
          const int jb = s.cell_start[nr], je = s.cell_start[nr + 1];
          for (int jj = jb; jj < je; ++jj) {
            const int j = s.members[jj];
            const int4 qj = s.q[j];
            if (!valid || j == i) continue;
            const float dx = (float)min_image_fixed(qi.x, qj.x) * fs0;
            const float dy = (float)min_image_fixed(qi.y, qj.y) * fs1;
            const float dz = (float)min_image_fixed(qi.z, qj.z) * fs2;
            const float r2 = dx * dx + dy * dy + dz * dz;
            const int p = ti * nt + qj.w;
            const float rl2 = rl2s[w][p];
            bool keep = r2 < rl2 * (1.0f - NL_BAND);
            if (!keep && r2 < rl2 * (1.0f + NL_BAND)) keep = exact_within(s, i, j, rl2d[w][p]);
            if (keep) {
              if (cnt < cap) row[cnt] = j;
              ++cnt;
            }
          }
        }
      }
    }
    if (valid) {
      s.nn[i] = cnt < cap ? cnt : cap;
      s.q_build[i] = qi;
      if (cnt > cap) {
        atomicMax(&s.flags->overflow_need, cnt);
        atomicCAS(&s.flags->error, 0, (int)DEV_OVERFLOW);
      }
      nb_sum += (unsigned long long)cnt;
    }
  }
  for (int o = 16; o > 0; o >>= 1) nb_sum += __shfl_down_sync(0xffffffffu, nb_sum, o);
  if (lane == 0 && nb_sum) atomicAdd(&s.flags->nb_total, nb_sum);
}

// ---- launch descriptors ----
#define SIMPLE_CALL(name, kern, block)                                           \
  KernelCall name(const SysDev* d, const Tile* tl, int ntiles, GroupCtl* ctl) { \
    KernelCall k = make_call((void*)kern, ntiles, block, 0);                    \
    put(k, d); put(k, tl); put(k, ctl);                                          \
    return k;                                                                    \
  }
SIMPLE_CALL(bin_call, k_bin, TILE_P)
SIMPLE_CALL(scan_call, k_scan, SCAN_THREADS)
SIMPLE_CALL(scatter_call, k_scatter, TILE_P)
SIMPLE_CALL(cellsort_call, k_cellsort, CELLS_PER_TILE * 32)
SIMPLE_CALL(permute_call, k_permute, TILE_P)
SIMPLE_CALL(copyback_call, k_copyback, TILE_P)
SIMPLE_CALL(nlist_call, k_nlist, CELLS_PER_TILE * 32)
#undef SIMPLE_CALL

}  // namespace gbmd
