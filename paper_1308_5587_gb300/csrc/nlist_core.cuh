// nlist_core.cuh -- the neighbour-list decision shared by the list builders (cell
// list in k_lists.cu, tree list in k_tree.cu): a pair is a neighbour when
// r^2 < r_list,ij^2, r_list,ij = r_cut,ij + r_buff (strict).  The builders test in
// FP32 on the exact fixed-point difference; a candidate within a relative band
// NL_BAND of r_list^2 is decided again in FP64, exactly as the reference
// definition computes it (the FP32 error is below 2e-6 relative).
#pragma once
#include "launch.cuh"

namespace gbmd {

constexpr float NL_BAND = 1e-5f;

// this step rebuilds the system's lists (decided by the last block of the step)
__device__ __forceinline__ bool rebuilding(const SysDev& s) {
  return ((const volatile Flags*)s.flags)->do_rebuild != 0;
}
// the same, read by one thread and shared with the block (every thread must call it)
__device__ __forceinline__ bool block_rebuilding(const SysDev& s) {
  __shared__ int r;
  if (threadIdx.x == 0) r = rebuilding(s);
  __syncthreads();
  return r != 0;
}
// launch counters: per system (the block of its first tile) and per group
__device__ __forceinline__ void count(const SysDev& s, const Tile& t, GroupCtl* ctl) {
  if (threadIdx.x == 0 && t.first == 0) atomicAdd(&s.flags->launches, 1ull);
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
}

// ---- FP64 decision for a candidate in the band: the reference definition ----
static __device__ __noinline__ bool exact_within(const SysDev& s, int i, int j, double rl2) {
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

}  // namespace gbmd
