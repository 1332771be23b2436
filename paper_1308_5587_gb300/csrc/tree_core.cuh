// tree_core.cuh -- the bounding-volume hierarchy of the tree neighbour list: node
// boxes, the periodic box-sphere test and the traversal order.  Plain C++ callable
// from host and device code, so that the same functions run inside the kernels
// (k_tree.cu) and in host-side checks.
//
// Section 5: HOOMD-blue builds neighbour lists for size-disperse systems with a
// bounding volume hierarchy (nlist.tree), one tree per particle type, each particle
// querying every type's tree with its own search radius.  Here the tree of a type is
// an implicit complete binary tree (heap numbering: root 1, children 2k and 2k + 1)
// over that type's particles in the order of the cell sort (Morton order of the cells,
// then of the particles inside a cell), TREE_LEAF particles per leaf; P leaves (P a
// power of two, the last ones empty).
// A node holds the axis-aligned box of its particles in 32-bit fixed point
// (u = q + 2^31 mod 2^32, i.e. the box [-L/2, L/2) mapped onto [0, 2^32)); an
// empty node has lo > hi on x.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define GBMD_HD __host__ __device__ __forceinline__
#else
#define GBMD_HD inline
#endif

namespace gbmd {

#ifndef GBMD_TREE_LEAF
#define GBMD_TREE_LEAF 4
#endif
constexpr int TREE_LEAF = GBMD_TREE_LEAF;   // particles per leaf

// node box: lo in (x, y, z), hi in (x2, y2, z2); 32 bytes, two 16-byte loads
struct alignas(16) TreeBox {
  uint32_t x, y, z, pad0;
  uint32_t x2, y2, z2, pad1;
};

GBMD_HD TreeBox tree_empty_box() {
  TreeBox b;
  b.x = b.y = b.z = 0xffffffffu;
  b.x2 = b.y2 = b.z2 = 0u;
  b.pad0 = b.pad1 = 0u;
  return b;
}

GBMD_HD bool tree_box_empty(const TreeBox& b) { return b.x > b.x2; }

GBMD_HD uint32_t tree_min(uint32_t a, uint32_t b) { return a < b ? a : b; }
GBMD_HD uint32_t tree_max(uint32_t a, uint32_t b) { return a > b ? a : b; }

// grow box b by the point (ux, uy, uz)
GBMD_HD void tree_box_add(TreeBox& b, uint32_t ux, uint32_t uy, uint32_t uz) {
  b.x = tree_min(b.x, ux); b.y = tree_min(b.y, uy); b.z = tree_min(b.z, uz);
  b.x2 = tree_max(b.x2, ux); b.y2 = tree_max(b.y2, uy); b.z2 = tree_max(b.z2, uz);
}

// the union of two boxes (an empty one adds nothing: its lo is all ones, hi zero)
GBMD_HD TreeBox tree_box_union(const TreeBox& a, const TreeBox& b) {
  TreeBox r;
  r.x = tree_min(a.x, b.x); r.y = tree_min(a.y, b.y); r.z = tree_min(a.z, b.z);
  r.x2 = tree_max(a.x2, b.x2); r.y2 = tree_max(a.y2, b.y2); r.z2 = tree_max(a.z2, b.z2);
  r.pad0 = r.pad1 = 0u;
  return r;
}

// Periodic distance, in fixed-point units, from coordinate u to the interval
// [lo, hi] (lo <= hi, no wrap) on the circle of circumference 2^32: zero inside,
// else the shorter way round to either end.  Never more than the minimum-image
// distance from u to any point of the interval.
GBMD_HD uint32_t tree_axis_gap(uint32_t u, uint32_t lo, uint32_t hi) {
  if (u - lo <= hi - lo) return 0u;
  const uint32_t up = lo - u, down = u - hi;
  return up < down ? up : down;
}

// squared distance (FP32, in length units) from the point to the node box
GBMD_HD float tree_gap2(const TreeBox& b, uint32_t ux, uint32_t uy, uint32_t uz, float fs0,
                        float fs1, float fs2) {
  const float gx = (float)tree_axis_gap(ux, b.x, b.x2) * fs0;
  const float gy = (float)tree_axis_gap(uy, b.y, b.y2) * fs1;
  const float gz = (float)tree_axis_gap(uz, b.z, b.z2) * fs2;
  return gx * gx + gy * gy + gz * gz;
}

// the node after node k's subtree in depth-first order (left child first): up past
// every right child (the trailing ones of k), then to the right sibling; 0 when the
// traversal is over
GBMD_HD int tree_next(int k) {
#if defined(__CUDA_ARCH__)
  const int ones = __ffs(~k) - 1;
#else
  const int ones = __builtin_ctz(~(unsigned)k);
#endif
  k >>= ones;
  return k ? k + 1 : 0;
}

// smallest power of two >= the leaves needed for n particles (at least 1)
GBMD_HD int tree_leaves(int n) {
  const int m = (n + TREE_LEAF - 1) / TREE_LEAF;
  int p = 1;
  while (p < m) p <<= 1;
  return p;
}

// Visit every leaf of the tree (boxes[1 .. 2P - 1], leaves at P .. 2P - 1) whose box
// lies within sqrt(r2) of the point: visit(leaf index b) for leaf node P + b.  At
// most max_nodes nodes are examined; returns the number examined, or -1 when that
// limit cut the traversal short.
template <class Visit>
GBMD_HD int tree_query(const TreeBox* boxes, int P, uint32_t ux, uint32_t uy, uint32_t uz,
                       float fs0, float fs1, float fs2, float r2, int max_nodes,
                       Visit&& visit) {
  int k = 1, seen = 0;
  while (k) {
    if (++seen > max_nodes) return -1;
    const TreeBox b = boxes[k];
    if (!tree_box_empty(b) && tree_gap2(b, ux, uy, uz, fs0, fs1, fs2) < r2) {
      if (k >= P) {
        visit(k - P);
      } else {
        k <<= 1;
        continue;
      }
    }
    k = tree_next(k);
  }
  return seen;
}

}  // namespace gbmd
