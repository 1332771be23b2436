// k_tree.cu -- the tree neighbour list (Section 5: nlist.tree, a bounding volume
// hierarchy per particle type, for size-disperse systems).
//
// After the cell sort (k_bin .. k_cellsort, type-major bins, Morton order of the
// particles inside a bin), type t's particles are members[tree_first[t] ..
// + tree_n[t]) in Morton order of cells, then of particles.  Its tree is the
// implicit complete binary tree of tree_core.cuh over them, TREE_LEAF particles per
// leaf.  Two kernels, both no-ops for systems not rebuilding or on the cell list:
//   k_tree_build  one thread per leaf: the leaf's box and a copy of its particles
//                 (position, index) in leaf order, then up the tree: the second child
//                 to arrive at a node writes its box (an arrival counter per node,
//                 which that child resets); no thread waits for another;
//   k_tree_nlist  one thread per particle, in cell order (neighbouring threads walk
//                 similar paths), the types with the longest queries first (they
//                 would otherwise finish last): for every type t, the leaves of t's
//                 tree within r_list(t_i, t) of the particle, then the same pair
//                 decision as the cell list (nlist_core.cuh).  The row holds the
//                 neighbours in (type, cell order) order.
// A traversal examines each node at most once, so 2 P nodes bound it; passing the
// bound (which cannot happen) would stop it and set DEV_TREE.
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

// fixed-point coordinate on [0, 2^32): the box [-L/2, L/2) in order
__device__ __forceinline__ uint32_t tree_u(int q) { return (uint32_t)q ^ 0x80000000u; }

// a node box written by another thread of this launch: from L2, past L1
__device__ __forceinline__ TreeBox load_box_l2(const TreeBox* p) {
  const uint4 a = __ldcg(reinterpret_cast<const uint4*>(p));
  const uint4 b = __ldcg(reinterpret_cast<const uint4*>(p) + 1);
  TreeBox r;
  r.x = a.x; r.y = a.y; r.z = a.z; r.pad0 = 0u;
  r.x2 = b.x; r.y2 = b.y; r.z2 = b.z; r.pad1 = 0u;
  return r;
}

__global__ void __launch_bounds__(TILE_P) k_tree_build(const SysDev* __restrict__ sysv,
                                                       const Tile* __restrict__ tiles,
                                                       GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  if (!rebuilding(s) || !s.tree || (int)threadIdx.x >= t.count) return;
  const int g = t.first + threadIdx.x;   // leaf number over all types of the system
  int ty = 0;
  while (ty + 1 < s.ntypes && g >= s.tree_leaf0[ty + 1]) ++ty;
  const int P = s.tree_P[ty], b = g - s.tree_leaf0[ty];
  TreeBox* boxes = s.tree_box + s.tree_node0[ty];
  unsigned* arrive = s.tree_arrive + s.tree_node0[ty];
  const int first = s.tree_first[ty], nty = s.tree_n[ty];
  const int4* __restrict__ qv = q_at(s, step_of(s.flags));
  TreeBox box = tree_empty_box();
#pragma unroll
  for (int k = 0; k < TREE_LEAF; ++k) {
    const int m = b * TREE_LEAF + k;
    if (m < nty) {
      const int j = s.members[first + m];
      const int4 q = qv[j];
      tree_box_add(box, tree_u(q.x), tree_u(q.y), tree_u(q.z));
      s.tree_q[first + m] = make_int4(q.x, q.y, q.z, j);   // the leaf's own copy
    }
  }
  int node = P + b;
  boxes[node] = box;
  while (node > 1) {   // at most log2(P) levels
    __threadfence();   // this thread's box before its arrival
    const int parent = node >> 1;
    if (atomicAdd(&arrive[parent], 1u) == 0u) return;   // the sibling goes on
    arrive[parent] = 0u;   // both children are in: ready for the next build
    __threadfence();
    box = tree_box_union(load_box_l2(boxes + 2 * parent), load_box_l2(boxes + 2 * parent + 1));
    boxes[parent] = box;
    node = parent;
  }
}

__global__ void __launch_bounds__(TILE_P) k_tree_nlist(const SysDev* __restrict__ sysv,
                                                       const Tile* __restrict__ tiles,
                                                       GroupCtl* ctl) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  count(s, t, ctl);
  if (!rebuilding(s) || !s.tree) return;   // uniform over the block
  const int nt = s.ntypes;
  __shared__ float thr_lo[MAXT2], thr_hi[MAXT2];
  __shared__ double rl2d[MAXT2];
  for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) {
    const float rl2 = s.pf[k].rl2;
    thr_lo[k] = rl2 * (1.0f - NL_BAND);
    thr_hi[k] = rl2 * (1.0f + NL_BAND);
    rl2d[k] = s.pd[k].rl2;
  }
  __syncthreads();
  const bool valid = (int)threadIdx.x < t.count;
  unsigned long long nb = 0;
  if (valid) {
    // launch position -> member: the types in the order of tree_qtype
    const int pos = t.first + threadIdx.x;
    int k = 0;
    while (k + 1 < nt && pos >= s.tree_qpos[k + 1]) ++k;
    const int ty = s.tree_qtype[k];
    const int i = s.members[s.tree_first[ty] + (pos - s.tree_qpos[k])];
    const int4* __restrict__ qv = q_at(s, step_of(s.flags));
    const int4 qi = qv[i];
    const uint32_t ux = tree_u(qi.x), uy = tree_u(qi.y), uz = tree_u(qi.z);
    const float fs0 = s.fscale[0], fs1 = s.fscale[1], fs2 = s.fscale[2];
    const int cap = s.cap, stride = s.nl_stride;
    int* __restrict__ nl = s.nl;
    int cnt = 0;
    bool cut = false;
    for (int tj = 0; tj < nt; ++tj) {
      const int p = qi.w * nt + tj;
      const float lo = thr_lo[p], hi = thr_hi[p];
      const double rl2 = rl2d[p];
      const int P = s.tree_P[tj], first = s.tree_first[tj], nty = s.tree_n[tj];
      const int seen = tree_query(
          s.tree_box + s.tree_node0[tj], P, ux, uy, uz, fs0, fs1, fs2, hi, 2 * P, [&](int b) {
            for (int k = 0; k < TREE_LEAF; ++k) {
              const int m = b * TREE_LEAF + k;
              if (m >= nty) break;
              const int4 qj = s.tree_q[first + m];
              const int j = qj.w;
              if (j == i) continue;
              const float dx = (float)min_image_fixed(qi.x, qj.x) * fs0;
              const float dy = (float)min_image_fixed(qi.y, qj.y) * fs1;
              const float dz = (float)min_image_fixed(qi.z, qj.z) * fs2;
              const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              if (r2 < hi && (r2 < lo || exact_within(s, i, j, rl2))) {
                nl[nl_index(i, min(cnt, cap - 1), stride)] = j;   // an overflowing row is rebuilt
                ++cnt;
              }
            }
          });
      cut |= seen < 0;
    }
    s.nn[i] = cnt < cap ? cnt : cap;
    s.q_build[i] = qi;
    if (cnt > cap) {
      atomicMax(&s.flags->overflow_need, cnt);
      atomicCAS(&s.flags->error, 0, (int)DEV_OVERFLOW);
    }
    if (cut) atomicCAS(&s.flags->error, 0, (int)DEV_TREE);
    nb = (unsigned long long)cnt;
  }
  for (int o = 16; o > 0; o >>= 1) nb += __shfl_down_sync(0xffffffffu, nb, o);
  if ((threadIdx.x & 31) == 0 && nb) atomicAdd(&s.flags->nb_total, nb);
}

KernelCall tree_build_call(const SysDev* d, const Tile* tiles_l, int ntiles, GroupCtl* ctl) {
  KernelCall k = make_call((void*)k_tree_build, ntiles, TILE_P, 0);
  put(k, d); put(k, tiles_l); put(k, ctl);
  return k;
}

KernelCall tree_nlist_call(const SysDev* d, const Tile* tiles_p, int ntiles, GroupCtl* ctl) {
  KernelCall k = make_call((void*)k_tree_nlist, ntiles, TILE_P, 0);
  put(k, d); put(k, tiles_p); put(k, ctl);
  return k;
}

}  // namespace gbmd
