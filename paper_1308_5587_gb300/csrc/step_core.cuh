// step_core.cuh -- the integration half of the fused step kernel (K5 + K6): the
// velocity-Verlet update of one particle once its force is known, and the end of
// the step (rebuild check, per-system decisions) done by the last block to finish.
//
// Velocity Verlet (Section 3.1 integrators; textbook form): with the stored velocity
// half a kick behind, step n of particle i is
//   v <- v + kick F_i(x^n),  kick = dt/m (closing half kick of step n-1 plus opening
//                            half kick of step n), or dt/(2m) right after create /
//                            set_state (v holds full-step velocities: Flags::v_full)
//   x <- x + dt v            (positions in box-fraction units x 2^32/L, so one FMA)
//   wrap into [-L/2, L/2), image += crossings, fixed-point shadow of x^{n+1}
// The shadows are double-buffered by step parity: the kernel of step n gathers
// neighbour positions from buffer n & 1 and writes x^{n+1} to the other one.
//
// FP64 runs at about 1/80 of the FP32 FMA rate on this part (measured: 1.6 against
// 128 FMAs per SM per clock), so the FP64 pipe only does the six FMAs of the kicks
// and drifts plus one add per axis: the FP32 force is widened to FP64 field by field
// on the integer pipe, and rint uses the 1.5 * 2^52 rounding constant.
#pragma once
#include "launch.cuh"

namespace gbmd {

// float -> double, exactly, on the integer pipe.  Zero and subnormal inputs (a
// force below 1.2e-38) give zero; inf / NaN set `bad`.
__device__ __forceinline__ double widen_f32(float f, bool& bad) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  bad |= ex == 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long mag = ((unsigned long long)(ex + 896u) << 52) |   // 1023 - 127
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)(sign | (ex ? mag : 0ull)));
}

// rint(x) (ties to even) as an integer for |x| < 2^51: x + 1.5 * 2^52 lies in
// [2^52, 2^53), where the spacing of doubles is 1, so the sum is rounded to an
// integer and its bit pattern minus the constant's is that integer
__device__ __forceinline__ long long rint_ll(double x) {
  const double m = x + 6755399441055744.0;
  return __double_as_longlong(m) - 0x4338000000000000LL;
}

// the lines of the particle's state that the integration reads, requested into L2
// before the force loop (no registers held through the loop)
__device__ __forceinline__ void prefetch_particle(const SysDev& s, int i) {
  const int n = s.n;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(s.x + a * n + i));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(s.v + a * n + i));
  }
  asm volatile("prefetch.global.L2 [%0];" ::"l"(s.q_build + i));
}

// the particle's state the integration reads
struct ParticleState {
  double v[3], xq[3];
  int4 qb;   // shadow at the last list build
};
__device__ __forceinline__ ParticleState load_particle(const SysDev& s, int i) {
  ParticleState p;
  const int n = s.n;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    p.v[a] = s.v[a * n + i];
    p.xq[a] = s.x[a * n + i];
  }
  p.qb = __ldg(s.q_build + i);
  return p;
}

// one particle's kick, drift, wrap and new shadow; `need` = it moved more than
// r_buff/2 since the last list build
template <int PREC>
__device__ __forceinline__ void integrate_one(const SysDev& s, int i, int ty, const double f[3],
                                              int vfull, const ParticleState& p0,
                                              int4* __restrict__ q_next,
                                              double4_32a* __restrict__ p64_next, bool& need,
                                              bool& bad) {
  const int n = s.n;
  if (s.n_ghost > 0 && __ldg(s.tag + i) >= n - s.n_ghost) {
    // a ghost (a copy of a particle another domain owns) keeps the position set
    // before the step: no kick, drift or displacement check; the next shadow repeats
    // the current one
    const int4 qg = make_int4((int)rint_ll(p0.xq[0]), (int)rint_ll(p0.xq[1]),
                              (int)rint_ll(p0.xq[2]), ty);
    q_next[i] = qg;
    if (PREC == GBMD_FP64)
      p64_next[i] = make_double4_32a(p0.xq[0] * (s.L[0] * (1.0 / 4294967296.0)),
                                     p0.xq[1] * (s.L[1] * (1.0 / 4294967296.0)),
                                     p0.xq[2] * (s.L[2] * (1.0 / 4294967296.0)),
                                     __longlong_as_double(ty));
    return;
  }
  const double kick = vfull ? s.h : s.h + s.h;
  double v[3], xq[3];
  int q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v[a] = fma(kick, f[a], p0.v[a]);
    xq[a] = fma(s.dtq[a], v[a], p0.xq[a]);
    long long qq = rint_ll(xq[a]);
    const long long k = (qq + 0x80000000LL) >> 32;       // floor((xq + 2^31) / 2^32)
    if (k != 0) {
      if (k > 1 || k < -1 || !isfinite(xq[a])) bad = true;
      xq[a] -= (double)k * 4294967296.0;
      qq -= k << 32;
      s.img[a * n + i] += (int)k;
    }
    q[a] = (int)qq;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s.v[a * n + i] = v[a];
    s.x[a * n + i] = xq[a];
  }
  q_next[i] = make_int4(q[0], q[1], q[2], ty);
  if (PREC == GBMD_FP64)
    p64_next[i] = make_double4_32a(xq[0] * (s.L[0] * (1.0 / 4294967296.0)),
                                   xq[1] * (s.L[1] * (1.0 / 4294967296.0)),
                                   xq[2] * (s.L[2] * (1.0 / 4294967296.0)),
                                   __longlong_as_double(ty));
  const float dx = (float)min_image_fixed(q[0], p0.qb.x) * s.fscale[0];
  const float dy = (float)min_image_fixed(q[1], p0.qb.y) * s.fscale[1];
  const float dz = (float)min_image_fixed(q[2], p0.qb.z) * s.fscale[2];
  need = dx * dx + dy * dy + dz * dz > s.rbuff_half2;
}

// NVT, first half at particle i once F_i(x^n) is known: the closing half kick and
// thermostat scaling of the previous step, u = (v + h F) exp(-xi dt/2) (just u = v
// right after create / set_state, when v holds full-step velocities); u is stored
// as the velocity and u.u returned for the kinetic energy.  The scale factor
// exp(-xi dt/2) is the one the previous step's opening half used (nh[2]).
__device__ __forceinline__ double nvt_close(const SysDev& s, int i, const double f[3], int vfull) {
  const int n = s.n;
  const double sc = s.nh[2];
  double uu = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double u = s.v[a * n + i];
    if (!vfull) u = fma(s.h, f[a], u) * sc;
    s.v[a * n + i] = u;
    uu = fma(u, u, uu);
  }
  return uu;
}

// FP64 sum over the block in a fixed order (warp shuffles, then the warps in order);
// the result is valid in thread 0
__device__ __forceinline__ double block_sum_fixed(double v) {
  __shared__ double wsum[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) wsum[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += wsum[k];
  __syncthreads();
  return t;
}

// End of the NVT force half, every block: publish this block's v.v partial sum and
// count the arrival; the last block updates every NVT system's thermostat
// (closing half of the previous step, then opening half of this one, with
// G = (2K/(g kT) - 1)/tau^2 at the kinetic energy K of the closing velocities):
//   eta += dt/2 xi;  xi += dt/2 G;     (skipped right after create / set_state)
//   xi += dt/2 G;    eta += dt/2 xi;   exp(-xi dt/2) for the opening scaling
__device__ __forceinline__ void nvt_half_tail(const SysDev& s, const SysDev* __restrict__ sysv,
                                              GroupCtl* ctl, int nsys, int total_blocks,
                                              double uu) {
  const double part = block_sum_fixed(uu);
  __shared__ int last;
  if (threadIdx.x == 0) {
    s.nh_part[blockIdx.x] = part;
    __threadfence();
    last = (atomicAdd(&ctl->blocks_done_a, 1u) == (unsigned)total_blocks - 1u);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int k = 0; k < nsys; ++k) {   // uniform over the block
    const SysDev& sk = sysv[k];
    if (!sk.nvt) continue;
    const FlagWords w = load_flag_words(sk.flags);
    const longlong2 sl = load_flag_pair(&sk.flags->step);
    if (!(w.error == 0 && (sl.y < 0 || sl.x < sl.y))) continue;
    double a = 0.0;   // this system's tiles, strided over the block in a fixed order
    for (int t = threadIdx.x; t < sk.tile_count_s; t += blockDim.x)
      a += ((const volatile double*)sk.nh_part)[sk.tile_first_s + t];
    const double sum = block_sum_fixed(a);
    if (threadIdx.x == 0) {
      const double K = 0.5 * sk.mass * sum;
      const double G = (2.0 * K / (sk.gdof * sk.kT) - 1.0) / (sk.tau * sk.tau);
      const double hdt = 0.5 * sk.dt;
      double xi = sk.nh[0], eta = sk.nh[1];
      if (!w.v_full) {
        eta += hdt * xi;
        xi += hdt * G;
      }
      xi += hdt * G;
      eta += hdt * xi;
      sk.nh[0] = xi;
      sk.nh[1] = eta;
      sk.nh[2] = exp(-hdt * xi);
    }
  }
  if (threadIdx.x == 0) ctl->blocks_done_a = 0;
}

// End of the step, every block of the step's force launches: publish this block's
// rebuild request / error, count the arrival; the last of `total_blocks` arrivals
// makes each system's decisions for the next step (step counter, rebuild, re-sort)
// and sets the CUDA-graph conditional of the rebuild.  No block waits on another.
__device__ __forceinline__ void step_tail(const SysDev& s, const SysDev* __restrict__ sysv,
                                          GroupCtl* ctl, int nsys, int total_blocks,
                                          cudaGraphConditionalHandle cond, int use_cond,
                                          bool need, bool bad) {
  const int any_need = __syncthreads_or(need);
  const int any_bad = __syncthreads_or(bad);
  __shared__ int last;
  if (threadIdx.x == 0) {
    if (any_bad) atomicCAS(&s.flags->error, 0, (int)DEV_NONFINITE);
    if (any_need) atomicOr(&s.flags->rebuild_req, 1);
    __threadfence();
    last = (atomicAdd(&ctl->blocks_done, 1u) == (unsigned)total_blocks - 1u);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  int any = 0;
  for (int k = threadIdx.x; k < nsys; k += blockDim.x) {
    Flags* gf = sysv[k].flags;
    volatile Flags* g = gf;
    // every field the decision needs, in flight together; then the stores
    const FlagWords w = load_flag_words(gf);
    const longlong2 sl = load_flag_pair(&gf->step);        // (step, step_limit)
    const longlong2 lr = load_flag_pair(&gf->last_sort);   // (last_sort, n_rebuilds)
    const long long nsort = g->n_sorts;
    const int sp = sysv[k].sort_period;
    const bool act = w.error == 0 && (sl.y < 0 || sl.x < sl.y);
    // a domain with ghosts only records the request: its caller rebuilds every domain
    const bool ext = sysv[k].n_ghost > 0;
    if (act) {
      const long long st = sl.x + 1;
      const int req = w.rebuild_req;
      const int rb = ext ? 0 : req;
      const int srt = rb && sp > 0 && (st - lr.x >= sp);
      g->step = st;
      g->v_full = 0;
      g->rebuild_req = ext ? req : 0;
      g->do_rebuild = rb;
      if (rb) g->n_rebuilds = lr.y + 1;
      if (srt) {
        g->last_sort = st;
        g->n_sorts = nsort + 1;
      }
      g->do_sort = srt;
      g->active = 1;
      any |= rb;
    } else {
      g->active = 0;
      g->do_rebuild = 0;
      g->do_sort = 0;
    }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    ctl->blocks_done = 0;
    ctl->any_rebuild = any;
    if (use_cond) cudaGraphSetConditional(cond, any ? 1u : 0u);
  }
}

}  // namespace gbmd
