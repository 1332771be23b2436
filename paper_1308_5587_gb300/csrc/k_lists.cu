// k_lists.cu -- cell list (integer binning + stable counting sort in Morton cell
// order), optional re-sort of the particle arrays, and the Verlet neighbour list.
//
// The paper names the structure (md.nlist.cell, Listing 1) and that HOOMD builds
// cell lists with atomic operations (Section 5); it gives no algorithm.  Here:
//   * a particle's cell comes from its 32-bit fixed-point coordinate, integer only:
//     c_a = floor((q_a + 2^31) * nc_a / 2^32), cell width L_a / nc_a >= r_list_max;
//   * cells are numbered by their rank in Morton (Z-order) of (cx, cy, cz);
//   * counting sort: atomic histogram -> exclusive scan -> atomic scatter, then
//     each cell's members are sorted by (the particle's own 30-bit Morton code,
//     index), so the result is the order (cell rank, fine Morton code, index)
//     whatever order the atomics ran in, and consecutive members of a cell are
//     spatial neighbours (a warp of the force kernel gathers from fewer lines:
//     2% off the step kernel at KA 10^6);
//   * neighbour list: full list (both i->j and j->i), one warp per cell whose lanes
//     are the cell's particles; every lane tests the same candidate j of the
//     neighbouring cells at a time (warp-uniform loop, broadcast loads).  Keep
//     j != i with r^2 < r_list,ij^2 (strict), r_list,ij = r_cut,ij + r_buff.  The
//     test runs in FP32 on the fixed-point difference; candidates within a relative
//     band of 1e-5 of r_list^2 are decided again in FP64 with the same operations
//     (and rounding) as the brute-force reference definition.  Hits are appended in
//     candidate order, so a row does not depend on how r^2 was rounded.
#include <algorithm>

#include "launch.cuh"
#include "nlist_core.cuh"

namespace gbmd {

KernelCall make_call(void* f, int grid, int block, size_t smem);

template <typename T>
static void put(KernelCall& k, const T& v) {
  static_assert(sizeof(T) <= 16, "arg too large");
  memcpy(k.store[k.nargs], &v, sizeof(T));
  ++k.nargs;
}

__device__ __forceinline__ bool sorting(const SysDev& s) {
  const FlagWords w = load_flag_words(s.flags);
  return w.do_rebuild != 0 && w.do_sort != 0;
}

// Morton code of the top 10 bits of each fixed-point coordinate (on [0, 2^32))
__device__ __forceinline__ unsigned spread10(unsigned v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__device__ __forceinline__ unsigned fine_morton(const int4& q) {
  return spread10(((unsigned)q.x ^ 0x80000000u) >> 22) |
         (spread10(((unsigned)q.y ^ 0x80000000u) >> 22) << 1) |
         (spread10(((unsigned)q.z ^ 0x80000000u) >> 22) << 2);
}

// The per-particle rebuild kernels (bin, scatter, permute, copyback) walk the tile
// table with a grid of at most WALK_BLOCKS blocks.  Warp 0 reads, for up to 32 of the
// block's next tiles at once, whether their system does this work (and counts the
// launch at each system's first tile); the block then works on those tiles only.  In
// a batch where a few members rebuild, the others' tiles then cost one parallel read,
// not a block each.
constexpr int WALK_BLOCKS = 152 * 8;

template <typename Active, typename Work>
__device__ __forceinline__ void walk_tiles(const SysDev* __restrict__ sysv,
                                           const Tile* __restrict__ tiles, int ntiles,
                                           GroupCtl* ctl, Active active, Work work) {
  __shared__ int act[32];
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
  for (int b0 = blockIdx.x; b0 < ntiles; b0 += 32 * gridDim.x) {
    __syncthreads();   // the previous round's act[] has been read
    if (threadIdx.x < 32) {
      const int b = b0 + threadIdx.x * gridDim.x;
      int a = 0;
      if (b < ntiles) {
        const Tile t = tiles[b];
        const SysDev& s = sysv[t.sys];
        if (t.first == 0) atomicAdd(&s.flags->launches, 1ull);
        a = active(s) ? 1 : 0;
      }
      act[threadIdx.x] = a;
    }
    __syncthreads();
    for (int l = 0; l < 32; ++l) {
      const int b = b0 + l * gridDim.x;
      if (b >= ntiles) break;
      if (!act[l]) continue;
      const Tile t = tiles[b];
      if ((int)threadIdx.x < t.count) work(sysv[t.sys], t.first + (int)threadIdx.x);
    }
  }
}

// ---- binning + histogram ----
__device__ __forceinline__ void bin_one(const SysDev& s, int i) {
  const int4 q = q_at(s, step_of(s.flags))[i];
  const int cx = cell_of_fixed(q.x, s.nc[0]);
  const int cy = cell_of_fixed(q.y, s.nc[1]);
  const int cz = cell_of_fixed(q.z, s.nc[2]);
  // the tree list sorts type-major (each type's particles contiguous, in cell order);
  // inside a bin every list orders by the particle's own Morton code
  const int r = s.lin2rank[(cz * s.nc[1] + cy) * s.nc[0] + cx] + (s.tree ? q.w * s.ncells : 0);
  s.key[i] = r;
  s.fkey[i] = fine_morton(q);
  // consecutive particles mostly share a bin: one atomic per distinct bin of the warp
  const unsigned am = __activemask();
  const unsigned peers = __match_any_sync(am, r);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&s.cell_cnt[r], __popc(peers));
}

__global__ void __launch_bounds__(TILE_P) k_bin(const SysDev* __restrict__ sysv,
                                                const Tile* __restrict__ tiles, int ntiles,
                                                GroupCtl* ctl) {
  walk_tiles(sysv, tiles, ntiles, ctl, [](const SysDev& s) { return rebuilding(s); }, bin_one);
}

// ---- exclusive scan of the bin counts (one block per system) ----
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
    s.flags->max_window = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nc = s.nbins;
  // four bins per thread (one 16-byte load where all four exist; the buffers come
  // from cudaMalloc, so 16-byte aligned)
  for (int base = 0; base < nc; base += 4 * SCAN_THREADS) {
    const int c = base + 4 * threadIdx.x;
    int v[4];
    if (c + 3 < nc) {
      const int4 q = *reinterpret_cast<const int4*>(s.cell_cnt + c);
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
      for (int k = 0; k < 4; ++k) v[k] = c + k < nc ? s.cell_cnt[c + k] : 0;
    }
    const int v4 = v[0] + v[1] + v[2] + v[3];
    int x = v4;
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
    int e[4];
    e[0] = carry + (wid ? warp_tot[wid - 1] : 0) + x - v4;
    e[1] = e[0] + v[0];
    e[2] = e[1] + v[1];
    e[3] = e[2] + v[2];
    if (c + 3 < nc) {
      const int4 q = make_int4(e[0], e[1], e[2], e[3]);
      *reinterpret_cast<int4*>(s.cell_start + c) = q;
      *reinterpret_cast<int4*>(s.cell_cursor + c) = q;
      *reinterpret_cast<int4*>(s.cell_cnt + c) = make_int4(0, 0, 0, 0);   // next build
    } else {
      for (int k = 0; k < 4; ++k) {
        if (c + k < nc) {
          s.cell_start[c + k] = e[k];
          s.cell_cursor[c + k] = e[k];
          s.cell_cnt[c + k] = 0;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) s.cell_start[nc] = carry;
}

// ---- scatter particle indices into their cells (unordered within a cell) ----
__global__ void __launch_bounds__(TILE_P) k_scatter(const SysDev* __restrict__ sysv,
                                                    const Tile* __restrict__ tiles, int ntiles,
                                                    GroupCtl* ctl) {
  walk_tiles(sysv, tiles, ntiles, ctl, [](const SysDev& s) { return rebuilding(s); },
             [](const SysDev& s, int i) {
               // one atomic per distinct bin of the warp; the peers take consecutive
               // slots after their leader's (the order inside a bin is fixed later)
               const int r = s.key[i];
               const int lane = threadIdx.x & 31;
               const unsigned am = __activemask();
               const unsigned peers = __match_any_sync(am, r);
               const int leader = __ffs(peers) - 1;
               int base = 0;
               if (lane == leader) base = atomicAdd(&s.cell_cursor[r], __popc(peers));
               base = __shfl_sync(am, base, leader);
               s.members_tmp[base + __popc(peers & ((1u << lane) - 1u))] = i;
             });
}

// ---- sort each bin's members (warp per bin) -> a deterministic order ----
// By (fine Morton code, index), so that consecutive members of a bin are spatial
// neighbours (the tree list's leaves; the force kernel's warps).
__global__ void __launch_bounds__(CELLS_PER_TILE * 32) k_cellsort(const SysDev* __restrict__ sysv,
                                                                  const Tile* __restrict__ tiles,
                                                                  GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!block_rebuilding(s) || w >= t.count) return;
  const int r = t.first + w;
  const int b = s.cell_start[r], e = s.cell_start[r + 1], n = e - b;
  // the sort key of member m: (fine code, index)
  auto key = [&](int v) -> unsigned long long {
    return ((unsigned long long)s.fkey[v] << 32) | (unsigned)v;
  };
  // the members' positions are copied in the same order: the list build then reads
  // a cell's candidates contiguously, however far the particles have drifted from
  // the order of the last re-sort
  const int4* __restrict__ qv = q_at(s, step_of(s.flags));
  if (n <= 32) {
    const int v = lane < n ? s.members_tmp[b + lane] : 0x7fffffff;
    const unsigned long long kv = lane < n ? key(v) : ~0ull;
    int rk = 0;
    for (int k = 0; k < 32; ++k) rk += __shfl_sync(0xffffffffu, kv, k) < kv;
    if (lane < n) {
      s.members[b + rk] = v;
      s.rmember[v] = b + rk;
      s.cpos[b + rk] = qv[v];
    }
  } else {
    for (int m = lane; m < n; m += 32) {
      const int v = s.members_tmp[b + m];
      const unsigned long long kv = key(v);
      int rk = 0;
      for (int k = 0; k < n; ++k) rk += key(s.members_tmp[b + k]) < kv;
      s.members[b + rk] = v;
      s.rmember[v] = b + rk;
      s.cpos[b + rk] = qv[v];
    }
  }
}

// ---- re-sort: gather every per-particle array into cell order ----
// Both kernels run at every rebuild and do work only when the system re-sorts (the
// tile walker makes that cheap when it does not).
__device__ __forceinline__ void permute_one(const SysDev& s, int k) {
  const int n = s.n;
  const int o = s.members[k];
  for (int a = 0; a < 3; ++a) {
    s.x_alt[a * n + k] = s.x[a * n + o];
    s.v_alt[a * n + k] = s.v[a * n + o];
    s.img_alt[a * n + k] = s.img[a * n + o];
  }
  s.type_alt[k] = s.type[o];
  s.tag_alt[k] = s.tag[o];
  s.q_alt[k] = q_at(s, step_of(s.flags))[o];
}

__device__ __forceinline__ void copyback_one(const SysDev& s, int k) {
  const int n = s.n;
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
  const long long step = step_of(s.flags);
  q_at(s, step)[k] = s.q_alt[k];
  s.members[k] = k;
  s.rmember[k] = k;
  if (s.precision == GBMD_FP64)
    p64_at(s, step)[k] = make_double4_32a(xr[0], xr[1], xr[2], __longlong_as_double(ty));
}

__global__ void __launch_bounds__(TILE_P) k_permute(const SysDev* __restrict__ sysv,
                                                    const Tile* __restrict__ tiles, int ntiles,
                                                    GroupCtl* ctl) {
  walk_tiles(sysv, tiles, ntiles, ctl, [](const SysDev& s) { return sorting(s); }, permute_one);
}

__global__ void __launch_bounds__(TILE_P) k_copyback(const SysDev* __restrict__ sysv,
                                                     const Tile* __restrict__ tiles, int ntiles,
                                                     GroupCtl* ctl) {
  walk_tiles(sysv, tiles, ntiles, ctl, [](const SysDev& s) { return sorting(s); }, copyback_one);
}

// ---- staged force tiles: the window of every aligned 2x2x2 block of cells ----
// One warp per block.  The window is the 4x4x4 cells around the block (the union
// of its cells' 27-cell stencils; distinct because every axis has >= 4 cells),
// listed with x fastest; each window cell contributes its member range, placed at
// a running offset.  The block's own cells have 8 consecutive Morton codes, so
// their members form one contiguous range.
__global__ void __launch_bounds__(256) k_blocks(const SysDev* __restrict__ sysv,
                                                const Tile* __restrict__ tiles, GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!rebuilding(s) || !s.staged || w >= t.count) return;
  const int b = t.first + w;
  const int nb0 = s.nb[0], nb1 = s.nb[1];
  const int bx = b % nb0, by = (b / nb0) % nb1, bz = b / (nb0 * nb1);
  const int nc0 = s.nc[0], nc1 = s.nc[1], nc2 = s.nc[2];
  int st[2], cn[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int wi = lane + 32 * h;
    const int cx = (2 * bx - 1 + (wi & 3) + nc0) % nc0;
    const int cy = (2 * by - 1 + ((wi >> 2) & 3) + nc1) % nc1;
    const int cz = (2 * bz - 1 + (wi >> 4) + nc2) % nc2;
    const int r = s.lin2rank[(cz * nc1 + cy) * nc0 + cx];
    st[h] = s.cell_start[r];
    cn[h] = s.cell_start[r + 1] - st[h];
  }
  int p0 = cn[0], p1 = cn[1];   // inclusive prefixes
  for (int o = 1; o < 32; o <<= 1) {
    const int y0 = __shfl_up_sync(0xffffffffu, p0, o);
    const int y1 = __shfl_up_sync(0xffffffffu, p1, o);
    if (lane >= o) {
      p0 += y0;
      p1 += y1;
    }
  }
  const int tot0 = __shfl_sync(0xffffffffu, p0, 31);
  const int wtot = tot0 + __shfl_sync(0xffffffffu, p1, 31);
  s.blk_win[(size_t)b * WIN_CELLS + lane] = make_int2(st[0], p0 - cn[0]);
  s.blk_win[(size_t)b * WIN_CELLS + 32 + lane] = make_int2(st[1], tot0 + p1 - cn[1]);
  // the block's own cells: lanes 0..7 take (ox, oy, oz)
  int rk = 0x7fffffff;
  bool exists = false;
  if (lane < 8) {
    const int cx = 2 * bx + (lane & 1), cy = 2 * by + ((lane >> 1) & 1), cz = 2 * bz + (lane >> 2);
    exists = cx < nc0 && cy < nc1 && cz < nc2;
    if (exists) rk = s.lin2rank[(cz * nc1 + cy) * nc0 + cx];
  }
  const int nown = __popc(__ballot_sync(0xffffffffu, exists));
  for (int o = 16; o > 0; o >>= 1) rk = min(rk, __shfl_xor_sync(0xffffffffu, rk, o));
  if (lane == 0) {
    const int first = s.cell_start[rk];
    s.blk_info[b] = make_int4(first, s.cell_start[rk + nown] - first, wtot, 0);
    atomicMax(&s.flags->max_window, wtot);
    if (wtot > s.window_cap) atomicCAS(&s.flags->error, 0, (int)DEV_WINDOW);
  }
}

// ---- neighbour list: one warp per cell ----
// Lanes are the cell's particles (up to 32 at a time).  The candidates -- the
// members of the stencil cells in (dz, dy, dx) cell order and member order within
// a cell, flattened into one stream, their positions read from the copy in cell
// order that the cell sort wrote -- pass through a per-warp shared-memory buffer
// 32 at a time, each converted once into FP32 coordinates relative to the centre
// of the warp's cell (the fixed-point difference takes care of the periodic wrap)
// plus j | type << 30; the next chunk is loaded while the current one is tested.
// Every lane then tests the broadcast candidate against its own particle with
// packed FP32x2 arithmetic (no integer work per test) and appends hits to its row,
// so each row holds its neighbours in (stencil cell, member) order.  Candidates
// within a relative band of 1e-5 of r_list^2 are decided in FP64 as the definition
// does (the FP32 error is below 2e-6 relative).
//
// With at least 3 cells per axis (REL) each chunk is first culled: a candidate
// farther than the largest r_list from the bounding box of the warp's particles
// cannot be anyone's neighbour, and the survivors are compacted (at KA density
// 44% of the stencil lies outside that reach).  The test yields two bit masks per
// lane -- r^2 below r_list^2 (1 - band), a neighbour, and below r_list^2 (1 + band)
// -- so appending a hit is a load of its index and a store, and only the rare
// candidates between the two go through the FP64 decision.  Hits are appended in
// candidate order either way, so a row is the same whichever variant built it.
constexpr int NL_TYPE_SHIFT = 30;
// REL rows of the global list: the final hit masks of up to NL_SEG tested chunks wait
// in shared memory, with their candidates in a ring of NL_JR indices, and each lane
// then appends all its hits of the segment in one loop (NL_JR >= 32 NL_SEG + 63: the
// tested segment plus the candidates compacted but not yet tested)
constexpr int NL_SEG = 14;
constexpr int NL_JR = 512;
static_assert(NL_JR >= 32 * NL_SEG + 63 && (NL_JR & (NL_JR - 1)) == 0, "segment ring");
// a culled candidate is at least this factor beyond the largest r_list^2 (1 + band)
// from the warp's box, far above the FP32 rounding of the box distance
constexpr float NL_CULL_MARGIN = 1e-4f;

// fixed-point coordinate of the centre of cell c of nc along an axis
__device__ __forceinline__ int cell_centre_fixed(int c, int nc) {
  const unsigned long long u = ((2ull * (unsigned long long)c + 1ull) << 32) / (2ull * (unsigned long long)nc);
  return (int)((unsigned int)u ^ 0x80000000u);
}

__device__ __forceinline__ float warp_min(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// distance of c from the interval [lo, hi] (0 inside)
__device__ __forceinline__ float gap_to(float c, float lo, float hi) {
  return fmaxf(fmaxf(lo - c, c - hi), 0.0f);
}
// shift the sign bit of v into the low end of m (candidate k of a chunk of mm
// ends at bit mm - 1 - k)
__device__ __forceinline__ unsigned push_sign(unsigned m, float v) {
  return __funnelshift_l(__float_as_uint(v), m, 1);
}

// With at least 3 cells on every axis, a candidate's coordinate relative to the cell
// centre, taken in [-L/2, L/2), is already its minimum image with respect to every
// particle of the cell (|d| < r_list <= w and the particle lies within w/2 of the
// centre).  With 1 or 2 cells on an axis a neighbour may sit on either side, so such
// a system keeps fixed-point coordinates and takes the minimum image per test.  The
// REL instance serves launches whose systems all have 3 cells per axis; the other
// decides per system.
template <bool MULTI, bool REL, bool STAGED>
__global__ void __launch_bounds__(CELLS_PER_TILE * 32, 3) k_nlist(const SysDev* __restrict__ sysv,
                                                                  const Tile* __restrict__ tiles,
                                                                  GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!block_rebuilding(s) || s.tree || w >= t.count) return;
  const int nt = s.ntypes;
  // r_list^2 (1 -+ band) per type pair (FP32)
  __shared__ float thr_lo[CELLS_PER_TILE][MAXT2], thr_hi[CELLS_PER_TILE][MAXT2];
  __shared__ double rl2d[CELLS_PER_TILE][MAXT2];
  // the chunk of candidates: x, y, z (relative to the cell centre; raw fixed point
  // without REL) and the type as 0/1, candidates 2m and 2m + 1 interleaved as
  // cxy[m] = (x, x', y, y') and czt[m] = (z, z', t, t') so that a pair loads as two
  // 16-byte words of FP32x2 operands; and j | type << 30
  __shared__ float4 cxy[CELLS_PER_TILE][32], czt[CELLS_PER_TILE][32];
  __shared__ int cjs[CELLS_PER_TILE][64];
  __shared__ int cand_l[STAGED ? CELLS_PER_TILE : 1][64];   // window-local index
  __shared__ float wbox[CELLS_PER_TILE][6];   // the pass's bounding box (culling)
  __shared__ int jring[CELLS_PER_TILE][NL_JR];             // j of kept candidates (REL)
  __shared__ unsigned hmask[CELLS_PER_TILE][NL_SEG][32];   // a lane's hits per chunk
  // STAGED: some member of the group may use the staged force path (decided per
  // system below); otherwise none does
  const bool staged = STAGED && s.staged != 0;   // then every axis has >= 4 cells
  float hi_max = 0.0f;
  for (int k = lane; k < nt * nt; k += 32) {
    const float rl2 = s.pf[k].rl2;
    thr_lo[w][k] = rl2 * (1.0f - NL_BAND);
    thr_hi[w][k] = rl2 * (1.0f + NL_BAND);
    rl2d[w][k] = s.pd[k].rl2;
    hi_max = fmaxf(hi_max, thr_hi[w][k]);
  }
  // culling radius^2 of a chunk (the largest r_list, with margin)
  const float cull2 = warp_max(hi_max) * (1.0f + NL_CULL_MARGIN);
  // r^2 - hi = (r^2 - lo) - (kappa - 1) lo, kappa = (1 + band) / (1 - band)
  const float km1 = 2.0f * NL_BAND / (1.0f - NL_BAND);
  const int r = t.first + w;
  const int nc0 = s.nc[0], nc1 = s.nc[1], nc2 = s.nc[2];
  const int lin = s.rank2lin[r];
  const int cx = lin % nc0, cy = (lin / nc0) % nc1, cz = lin / (nc0 * nc1);
  const int ox = cell_centre_fixed(cx, nc0), oy = cell_centre_fixed(cy, nc1),
            oz = cell_centre_fixed(cz, nc2);
  const float fs0 = s.fscale[0], fs1 = s.fscale[1], fs2 = s.fscale[2];
  // distinct neighbour-cell offsets per axis (fewer than 3 cells: no duplicates)
  const int lo0 = nc0 >= 3 ? -1 : 0, n0 = nc0 >= 3 ? 3 : nc0;
  const int lo1 = nc1 >= 3 ? -1 : 0, n1 = nc1 >= 3 ? 3 : nc1;
  const int lo2 = nc2 >= 3 ? -1 : 0, n2 = nc2 >= 3 ? 3 : nc2;
  const int nsc = n0 * n1 * n2;   // <= 27
  // REL: every system of the launch has >= 3 cells per axis; otherwise each system
  // takes the relative-coordinate path when it has them (warp-uniform: a warp is one
  // cell of one system), so a batch with one small member builds the others fast
  const bool rel = REL || (nc0 >= 3 && nc1 >= 3 && nc2 >= 3);
  const int own_sc = -lo0 + n0 * (-lo1 + n1 * -lo2);   // the cell's own stencil slot
  int sc_start = 0, sc_cnt = 0, sc_woff = 0;
  if (lane < nsc) {
    const int dx = lo0 + lane % n0, dy = lo1 + (lane / n0) % n1, dz = lo2 + lane / (n0 * n1);
    const int x = (cx + dx + nc0) % nc0, y = (cy + dy + nc1) % nc1, z = (cz + dz + nc2) % nc2;
    const int nr = s.lin2rank[(z * nc1 + y) * nc0 + x];
    sc_start = s.cell_start[nr];
    sc_cnt = s.cell_start[nr + 1] - sc_start;
    if (staged) {   // this stencil cell's place in the block's 4x4x4 window
      const int blk = ((cz >> 1) * s.nb[1] + (cy >> 1)) * s.nb[0] + (cx >> 1);
      const int wi = (((cz & 1) + 1 + dz) * 4 + ((cy & 1) + 1 + dy)) * 4 + ((cx & 1) + 1 + dx);
      sc_woff = s.blk_win[(size_t)blk * WIN_CELLS + wi].y;
    }
  }
  int incl = sc_cnt;   // inclusive prefix of the stencil cells' sizes
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int excl = incl - sc_cnt;
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const int b = s.cell_start[r], e = s.cell_start[r + 1];
  const int cap = s.cap;
  const int* __restrict__ members = s.members;
  const int4* __restrict__ cpos = s.cpos;   // member m's position (written by the cell sort)
  const bool two = !MULTI || nt <= 2;
  __syncwarp();

  auto put_cand = [&](int sl, float x, float y, float z, float t) {
    float* a = reinterpret_cast<float*>(&cxy[w][sl >> 1]) + (sl & 1);
    float* c = reinterpret_cast<float*>(&czt[w][sl >> 1]) + (sl & 1);
    a[0] = x;
    a[2] = y;
    c[0] = z;
    c[2] = t;
  };
  // component a (0 x, 1 y, 2 z) of slot sl
  auto cand_comp = [&](int sl, int a) -> float {
    const float* b = reinterpret_cast<const float*>(a < 2 ? &cxy[w][sl >> 1] : &czt[w][sl >> 1]);
    return b[(a == 1 ? 2 : 0) + (sl & 1)];
  };

  // candidate c of the flattened stream into registers (every lane runs every
  // shuffle); written to the chunk arrays by stage() once the previous chunk is done
  int4 nq = make_int4(0, 0, 0, 0);   // w = j | type << 30 (types 2, 3 set the sign bit)
  bool nempty = true;                // past the end of the stream
  int nloc = 0;
  auto fetch = [&](int c) {
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int mid = lo + step;
      const int v = __shfl_sync(0xffffffffu, excl, mid & 31);
      if (mid < nsc && c >= v) lo = mid;
    }
    const int st = __shfl_sync(0xffffffffu, sc_start, lo);
    const int ex = __shfl_sync(0xffffffffu, excl, lo);
    if (STAGED) nloc = __shfl_sync(0xffffffffu, sc_woff, lo) + (c - ex);
    nempty = c >= total;
    if (nempty) {
      nq = make_int4(0, 0, 0, 0);
      return;
    }
    const int j = members[st + (c - ex)];
    const int4 qj = cpos[st + (c - ex)];
    nq = make_int4(qj.x, qj.y, qj.z, j | (qj.w << NL_TYPE_SHIFT));
  };

  unsigned long long nb_sum = 0;
  for (int ibase = b; ibase < e; ibase += 32) {
    const bool valid = ibase + lane < e;
    const int i = valid ? members[ibase + lane] : -1;
    const int4 qi = valid ? cpos[ibase + lane] : make_int4(0, 0, 0, 0);
    const float xi = (float)min_image_fixed(qi.x, ox) * fs0;
    const float yi = (float)min_image_fixed(qi.y, oy) * fs1;
    const float zi = (float)min_image_fixed(qi.z, oz) * fs2;
    const float2 nX = make_float2(-xi, -xi), nY = make_float2(-yi, -yi), nZ = make_float2(-zi, -zi);
    // the bounding box of this pass's particles (REL culling)
    // (kept in shared memory: read once per fetched chunk, they need no registers)
    {
      const float bx0 = warp_min(valid ? xi : 3e38f), bx1 = warp_max(valid ? xi : -3e38f);
      const float by0 = warp_min(valid ? yi : 3e38f), by1 = warp_max(valid ? yi : -3e38f);
      const float bz0 = warp_min(valid ? zi : 3e38f), bz1 = warp_max(valid ? zi : -3e38f);
      if (lane == 0) {
        wbox[w][0] = bx0; wbox[w][1] = bx1; wbox[w][2] = by0;
        wbox[w][3] = by1; wbox[w][4] = bz0; wbox[w][5] = bz1;
      }
      __syncwarp();
    }
    // An idle lane gets thresholds -1 (never keeps).  Two types: -lo for a type-0
    // candidate and its change for type 1 in registers; more types read the table.
    const int pt = MULTI ? qi.w * nt : 0;
    const float lo_0 = valid ? thr_lo[w][pt] : -1.0f;
    const float lo_1 = valid && MULTI ? thr_lo[w][pt + min(1, nt - 1)] : lo_0;
    const float2 nl0 = make_float2(-lo_0, -lo_0), ndl = make_float2(lo_0 - lo_1, lo_0 - lo_1);
    const float2 k2 = make_float2(km1, km1);
    const int stride = s.nl_stride;
    const int i_row = valid ? i : 0;
    int cnt = 0;
    // the row's next ELL4 entry: entry k at row + (k / 4) * 4 stride + k % 4
    int* wp = s.nl + (size_t)i_row * 4;
    const size_t step4 = (size_t)stride * 4 - 3;
    const int m_row = ibase + lane;   // member rank (staged list rows)
    unsigned short* __restrict__ nl16 = reinterpret_cast<unsigned short*>(s.nl);
    // the particle's own place in the candidate stream (its cell is stencil cell
    // own_sc; a pass covers members ibase .. ibase + 31 of that cell)
    const int self_pos = __shfl_sync(0xffffffffu, excl, own_sc) + (ibase - b) + lane;

    // Hits of the 32 candidates at ring slots hb .. hb + 31: candidate k at bit 31 - k
    // of mlo (r^2 below lo: a neighbour) and mhi (below hi: a neighbour or within the
    // band).  The band is decided in FP64 first; then the hits are appended in
    // candidate order (the row does not depend on how r^2 was rounded).  Entries
    // past the capacity are counted, not stored.
    auto resolve_band = [&](unsigned mlo, unsigned mhi, int hb) -> unsigned {
      unsigned band = mhi & ~mlo;
      while (band) {
        const int k = __clz(band);
        band &= 0x7fffffffu >> k;
        const int cw = cjs[w][hb + k];
        const int j = cw & ((1 << NL_TYPE_SHIFT) - 1);
        const int p = MULTI ? pt + ((unsigned)cw >> NL_TYPE_SHIFT) : 0;
        if (!exact_within(s, i, j, rl2d[w][p])) mhi &= ~(0x80000000u >> k);
      }
      return mhi;
    };
    auto append_hits = [&](unsigned mlo, unsigned mhi, int hb) {
      mhi = resolve_band(mlo, mhi, hb);
      if (!staged) {
        const int* __restrict__ cj = &cjs[w][hb];
        while (mhi) {
          const int k = __clz(mhi);
          mhi &= 0x7fffffffu >> k;
          const int j = cj[k] & ((1 << NL_TYPE_SHIFT) - 1);
          if (cnt < cap) *wp = j;
          ++cnt;
          wp += (cnt & 3) ? 1 : step4;
        }
      } else {
        while (mhi) {
          const int k = __clz(mhi);
          mhi &= 0x7fffffffu >> k;
          if (cnt < cap) nl16[nl16_index(m_row, cnt, stride)] = (unsigned short)cand_l[w][hb + k];
          ++cnt;
        }
      }
    };

    // The deferred append of a segment (REL, global rows): chunk c's final mask of
    // this lane is hmask[c], bit c of nzb says it is not empty.  Hits are taken in
    // (chunk, candidate) order, four to a 16-byte store of the row's next slot group
    // (a short last group is padded with its first entry, which lies past the count
    // unless the next segment overwrites it).
    int4* __restrict__ nl4 = reinterpret_cast<int4*>(s.nl) + i_row;
    unsigned nzb = 0;
    int nseg = 0, seg0 = 0;
    auto flush = [&]() {
      unsigned m = 0;
      int c = 0;
      auto next = [&](int& j) -> bool {
        if (m == 0u) {
          if (nzb == 0u) return false;
          c = __ffs(nzb) - 1;
          nzb &= nzb - 1u;
          m = hmask[w][c][lane];
        }
        const int k = __clz(m);
        m &= 0x7fffffffu >> k;
        j = jring[w][(seg0 + c * 32 + k) & (NL_JR - 1)];
        return true;
      };
      int j0, j1, j2, j3;
      while ((cnt & 3) != 0 && next(j0)) {   // complete the group the last segment began
        if (cnt < cap) s.nl[((size_t)(cnt >> 2) * stride + i_row) * 4 + (cnt & 3)] = j0;
        ++cnt;
      }
      for (;;) {
        if (!next(j0)) break;
        int r = 1;
        j1 = j2 = j3 = j0;
        if (next(j1)) {
          ++r;
          if (next(j2)) {
            ++r;
            if (next(j3)) ++r;
          }
        }
        if (cnt < cap) nl4[(size_t)(cnt >> 2) * stride] = make_int4(j0, j1, j2, j3);
        cnt += r;
        if (r < 4) break;
      }
      nseg = 0;
    };

    fetch(lane);
    if (rel) {
      // Kept candidates go into a ring of 64 slots in stream order; every time 32
      // are waiting they are tested together (a full, unrolled chunk), so culling
      // saves tests and not only stores.  The particle's own candidate is always
      // kept (it lies in the box); selfabs is its ring position.
      int fill = 0, tested = 0, selfabs = -1;
      auto test32 = [&](int hb) {
        unsigned mlo = 0u, mhi = 0u;
#pragma unroll
        for (int k = 0; k < 32; k += 2) {
          const float4 A = cxy[w][(hb + k) >> 1];
          const float4 B = czt[w][(hb + k) >> 1];
          const float2 X = make_float2(A.x, A.y), Y = make_float2(A.z, A.w), Z = make_float2(B.x, B.y);
          float2 nlo;   // -r_list^2 (1 - band) of each candidate's type pair
          if (!MULTI) {
            nlo = nl0;
          } else if (two) {
            nlo = __ffma2_rn(make_float2(B.z, B.w), ndl, nl0);
          } else {
            const unsigned t0 = (unsigned)cjs[w][hb + k] >> NL_TYPE_SHIFT;
            const unsigned t1 = (unsigned)cjs[w][hb + k + 1] >> NL_TYPE_SHIFT;
            nlo = valid ? make_float2(-thr_lo[w][pt + (t0 & 3)], -thr_lo[w][pt + (t1 & 3)])
                        : make_float2(1.0f, 1.0f);
          }
          const float2 dx = __fadd2_rn(X, nX), dy = __fadd2_rn(Y, nY), dz = __fadd2_rn(Z, nZ);
          float2 d = __ffma2_rn(dx, dx, nlo);
          d = __ffma2_rn(dy, dy, d);
          d = __ffma2_rn(dz, dz, d);                  // r^2 - lo
          const float2 dh = __ffma2_rn(nlo, k2, d);   // r^2 - hi
          mlo = push_sign(push_sign(mlo, d.x), d.y);
          mhi = push_sign(push_sign(mhi, dh.x), dh.y);
        }
        const int rs = selfabs - tested;
        if (rs >= 0 && rs < 32) {
          mlo &= ~(0x80000000u >> rs);
          mhi &= ~(0x80000000u >> rs);
        }
        if (staged) {
          append_hits(mlo, mhi, hb);
        } else {
          if (nseg == 0) seg0 = tested;
          const unsigned m = resolve_band(mlo, mhi, hb);
          hmask[w][nseg][lane] = m;
          nzb |= (m != 0u ? 1u : 0u) << nseg;
          if (++nseg == NL_SEG) flush();
        }
      };
      for (int cb = 0; cb < total; cb += 32) {
        // relative coordinates; cull against the box and compact the survivors
        const float qx = (float)min_image_fixed(nq.x, ox) * fs0;
        const float qy = (float)min_image_fixed(nq.y, oy) * fs1;
        const float qz = (float)min_image_fixed(nq.z, oz) * fs2;
        const float gx = gap_to(qx, wbox[w][0], wbox[w][1]), gy = gap_to(qy, wbox[w][2], wbox[w][3]),
                    gz = gap_to(qz, wbox[w][4], wbox[w][5]);
        const bool keep = !nempty && fmaf(gz, gz, fmaf(gy, gy, gx * gx)) < cull2;
        const unsigned kb = __ballot_sync(0xffffffffu, keep);
        const int p = fill + __popc(kb & ((1u << lane) - 1u));
        if (keep) {
          const int sl = p & 63;
          put_cand(sl, qx, qy, qz, (float)(((unsigned)nq.w >> NL_TYPE_SHIFT) & 1u));
          cjs[w][sl] = nq.w;
          jring[w][p & (NL_JR - 1)] = nq.w & ((1 << NL_TYPE_SHIFT) - 1);
          if (STAGED) cand_l[w][sl] = nloc;
        }
        const int rs = self_pos - cb;
        if (rs >= 0 && rs < 32) selfabs = fill + __popc(kb & ((1u << rs) - 1u));
        fill += __popc(kb);
        __syncwarp();
        if (cb + 32 < total) fetch(cb + 32 + lane);   // in flight during the tests
        if (fill - tested >= 32) {
          test32(tested & 63);
          tested += 32;
        }
        __syncwarp();
      }
      if (fill > tested) {   // the last, partial chunk: pad it with far-away slots
        if (lane >= fill - tested) {
          const int sl = (tested + lane) & 63;
          put_cand(sl, 1e18f, 1e18f, 1e18f, 0.0f);
          cjs[w][sl] = 0;
        }
        __syncwarp();
        test32(tested & 63);
        __syncwarp();
      }
      if (nseg > 0) flush();
    } else {
      for (int cb = 0; cb < total; cb += 32) {
        put_cand(lane, __int_as_float(nq.x), __int_as_float(nq.y), __int_as_float(nq.z), 0.0f);
        cjs[w][lane] = nq.w;
        if (STAGED) cand_l[w][lane] = nloc;
        const int m = min(32, total - cb);
        __syncwarp();
        if (cb + 32 < total) fetch(cb + 32 + lane);   // in flight during the tests
        unsigned mlo = 0, mhi = 0;
        for (int k = 0; k < 32; ++k) {
          float r2 = 3e38f;
          int p = 0;
          if (k < m) {
            const float dx = (float)min_image_fixed(qi.x, __float_as_int(cand_comp(k, 0))) * fs0;
            const float dy = (float)min_image_fixed(qi.y, __float_as_int(cand_comp(k, 1))) * fs1;
            const float dz = (float)min_image_fixed(qi.z, __float_as_int(cand_comp(k, 2))) * fs2;
            r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const unsigned ct = (unsigned)cjs[w][k] >> NL_TYPE_SHIFT;
            p = !MULTI ? 0 : two ? (int)(ct & 1) : (int)ct;
          }
          const float lo = valid ? thr_lo[w][pt + p] : -1.0f;
          const float hi = valid ? thr_hi[w][pt + p] : -1.0f;
          mlo = (mlo << 1) | (r2 < lo ? 1u : 0u);
          mhi = (mhi << 1) | (r2 < hi ? 1u : 0u);
        }
        const int rs = self_pos - cb;
        if (rs >= 0 && rs < 32) {
          mlo &= ~(0x80000000u >> rs);
          mhi &= ~(0x80000000u >> rs);
        }
        append_hits(mlo, mhi, 0);
        __syncwarp();
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
SIMPLE_CALL(scan_call, k_scan, SCAN_THREADS)
SIMPLE_CALL(cellsort_call, k_cellsort, CELLS_PER_TILE * 32)
#define WALK_CALL(name, kern)                                                  \
  KernelCall name(const SysDev* d, const Tile* tl, int ntiles, GroupCtl* ctl) { \
    KernelCall k = make_call((void*)kern, std::min(ntiles, WALK_BLOCKS), TILE_P, 0);   \
    put(k, d); put(k, tl); put(k, ntiles); put(k, ctl);                            \
    return k;                                                                    \
  }
WALK_CALL(bin_call, k_bin)
WALK_CALL(scatter_call, k_scatter)
WALK_CALL(permute_call, k_permute)
WALK_CALL(copyback_call, k_copyback)
#undef WALK_CALL
SIMPLE_CALL(blocks_call, k_blocks, 256)
#undef SIMPLE_CALL

KernelCall nlist_call(const SysDev* d, const Tile* tl, int ntiles, GroupCtl* ctl, bool rel,
                      bool multi, bool staged) {
  void* const fs[2][2][2] = {
      {{(void*)k_nlist<false, false, false>, (void*)k_nlist<false, false, true>},
       {(void*)k_nlist<false, true, false>, (void*)k_nlist<false, true, true>}},
      {{(void*)k_nlist<true, false, false>, (void*)k_nlist<true, false, true>},
       {(void*)k_nlist<true, true, false>, (void*)k_nlist<true, true, true>}}};
  void* f = fs[multi ? 1 : 0][rel ? 1 : 0][staged ? 1 : 0];
  KernelCall k = make_call(f, ntiles, CELLS_PER_TILE * 32, 0);
  put(k, d); put(k, tl); put(k, ctl);
  return k;
}

}  // namespace gbmd
