// k_force.cuh -- the pair-force gather over the full Verlet neighbour list (K5),
// templated on the pair evaluator; each evaluator's variants are instantiated in
// their own translation unit (k_force.cu: LJ and WCA; k_force_mie.cu,
// k_force_yukawa.cu, k_force_gauss.cu).
//
// Section 3.1 / Listing 1: md.pair.lj(r_cut) with per type-pair epsilon, sigma, and
// the other short-range pair potentials listed beside it (Mie, WCA, Yukawa,
// Gaussian); Section 5 names the GPU technique: several threads per particle with
// warp-level reductions.  The paper gives no formula; the kernel computes, for every
// listed neighbour j of particle i with r^2 < r_cut,ij^2 (strict):
//   F_i += f(r) d_ij,  d_ij = x_i - x_j (minimum image),
// and optionally u_i += 1/2 (V(r) - V(r_cut)) and W_i,ab += 1/2 d_a f d_b, whose
// per-tile sums are reduced in FP64 together with the sum of v_i . v_i (kinetic
// energy, from the full-step velocity).  f and V per potential are in gbmd.h; for
// LJ, f = 24 eps [2 (sigma/r)^12 - (sigma/r)^6] / r^2.
//
// List layout (ELL4): entry k of particle i is nl[((k / 4) * stride + i) * 4 + k % 4]
// with stride = N rounded up to 32, so one int4 holds 4 consecutive entries of one
// particle and the int4s of consecutive particles are adjacent: a warp reading slot
// group g of 32 particles reads 512 contiguous bytes.
//
// Mapping: TPP (1, 2 or 4) lanes per particle; lane h takes slot groups h, h+TPP, ...
// The next slot group is fetched before the current one is used, and the four
// gathers of a group are in flight together.  Partial sums of the TPP lanes are
// combined with xor shuffles in a fixed order (deterministic).
//
// MIXED: positions come from the 32-bit fixed-point shadow q (int4: x, y, z, type).
// The int32 difference of two fixed-point coordinates is the minimum-image
// displacement exactly; it is converted to FP32 and scaled by L/2^32.  The pair
// arithmetic runs two neighbours at a time (LJ in packed FP32x2 operations); the
// per-particle sums are FP32.
// FP64: positions come from the double4 shadow p64; the minimum image is one
// conditional correction by L (|d| < L for wrapped coordinates); all arithmetic FP64.
#pragma once
#include "launch.cuh"
#include "step_core.cuh"
#include "fp64_math.cuh"

namespace gbmd {

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int TPP, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = TPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP64 block reduction of NPART per-particle values into partials[tile][0..7]
// (fixed order)
constexpr int NPART = 8;   // energy, virial xx xy xz yy yz zz, sum of v^2
template <int TPP, int BLOCK_MAX>
__device__ void reduce_partials(const double* vals, double* out) {
  constexpr int GMAX = BLOCK_MAX / TPP;
  __shared__ double sh[NPART][GMAX];
  const int g = threadIdx.x / TPP, l = threadIdx.x % TPP;
  const int ng = blockDim.x / TPP;
  if (l == 0)
    for (int c = 0; c < NPART; ++c) sh[c][g] = vals[c];
  __syncthreads();
  if (threadIdx.x < NPART) {
    double acc = 0;
    for (int k = 0; k < ng; ++k) acc += sh[threadIdx.x][k];
    out[threadIdx.x] = acc;
  }
}

// v_i . v_i at full step: the stored velocity is half a kick (h F_i) behind unless
// v_full (and, NVT, before the closing thermostat scaling); F_i is the force just
// computed (bitwise the stepping kernel's)
__device__ __forceinline__ double vsq(const SysDev& s, int i, double fx, double fy, double fz,
                                      int vfull) {
  const size_t n = (size_t)s.n;
  double v0 = s.v[i], v1 = s.v[n + i], v2 = s.v[2 * n + i];
  if (!vfull) {
    v0 = fma(s.h, fx, v0);
    v1 = fma(s.h, fy, v1);
    v2 = fma(s.h, fz, v2);
    if (s.nvt) {   // NVT: and the closing thermostat scaling (the opening one's factor)
      const double sc = s.nh[2];
      v0 *= sc;
      v1 *= sc;
      v2 *= sc;
    }
  }
  return v0 * v0 + v1 * v1 + v2 * v2;
}

// ---- pair evaluators: f (F_ij = f d_ij) and, with EV, the shifted energy v at r^2.
// The coefficients are those of PairF / PairD (gbmd_internal.cuh).  r^2 = 0 (an
// empty slot) may give inf or NaN: the caller's select drops it.

// FP32, one neighbour (the evaluators with transcendental functions)
template <int EVAL, bool EV>
__device__ __forceinline__ float eval_f32(float r2, const PairF& P, float& v) {
  if constexpr (EVAL == EVAL_MIE) {
    // (sigma/r)^n = 2^((n/2) log2(sigma^2/r^2)); one logarithm serves both powers
    const float r2i = rcp_approx(r2);
    const float lx = __log2f(P.p0 * r2i);
    const float tn = exp2f(P.p1 * lx), tm = exp2f(P.p2 * lx);
    if (EV) v = P.p3 * (tn - tm) - P.shift;
    return 2.f * P.p3 * (P.p1 * tn - P.p2 * tm) * r2i;
  } else if constexpr (EVAL == EVAL_YUKAWA) {
    const float ri = rsqrtf(r2);
    const float r = r2 * ri;
    const float e = P.p0 * __expf(-P.p1 * r) * ri;   // eps exp(-kappa r) / r
    if (EV) v = e - P.shift;
    return e * fmaf(P.p1, r, 1.f) * (ri * ri);
  } else {   // EVAL_GAUSS
    const float e = __expf(-P.p1 * r2);
    if (EV) v = P.p0 * e - P.shift;
    return P.p2 * e;
  }
}

// FP32x2: two neighbours; LJ in packed FP32x2 operations, the others per lane
template <int EVAL, bool EV>
__device__ __forceinline__ void eval_f32x2(const float2 r2, const PairF& Pa, const PairF& Pb,
                                           float2& f, float2& v) {
  if constexpr (EVAL == EVAL_LJ) {
    const float2 r2i = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
    const float2 r6i = __fmul2_rn(__fmul2_rn(r2i, r2i), r2i);
    const float2 lj1 = make_float2(Pa.p0, Pb.p0), mlj2 = make_float2(-Pa.p1, -Pb.p1);
    f = __fmul2_rn(__fmul2_rn(r2i, r6i), __ffma2_rn(lj1, r6i, mlj2));
    if (EV) {
      const float2 c12 = make_float2(Pa.p3, Pb.p3), mc6 = make_float2(-Pa.p4, -Pb.p4);
      const float2 msh = make_float2(-Pa.shift, -Pb.shift);
      v = __ffma2_rn(r6i, __ffma2_rn(c12, r6i, mc6), msh);
    }
  } else {
    f.x = eval_f32<EVAL, EV>(r2.x, Pa, v.x);
    f.y = eval_f32<EVAL, EV>(r2.y, Pb, v.y);
  }
}

// The FP64 path's FP32 pre-test keeps every pair with r^2 < r_cut^2 (1 + 1e-5): its
// FP32 r^2 (int32 difference, two roundings) is within 3e-7 relative of the FP64
// one, and the fixed-point shadow within 2^-32 L of the FP64 position.
constexpr float FP64_PRETEST_MARGIN = 1.0f + 1e-5f;

// FP64, one neighbour
template <int EVAL, bool EV>
__device__ __forceinline__ double eval_f64(double r2, const PairD& P, double& v) {
  if constexpr (EVAL == EVAL_LJ) {
    const double r2i = rcp_f64(r2);
    const double r6i = r2i * r2i * r2i;
    if (EV) v = fma(r6i, fma(P.p3, r6i, -P.p4), -P.shift);
    return r2i * r6i * fma(P.p0, r6i, -P.p1);
  } else if constexpr (EVAL == EVAL_MIE) {
    const double r2i = rcp_f64(r2);
    const double x = P.p0 * r2i;   // (sigma / r)^2
    const double tn = pow(x, P.p1), tm = pow(x, P.p2);
    if (EV) v = P.p3 * (tn - tm) - P.shift;
    return 2.0 * P.p3 * (P.p1 * tn - P.p2 * tm) * r2i;
  } else if constexpr (EVAL == EVAL_YUKAWA) {
    const double r = sqrt(r2);
    const double e = P.p0 * exp(-P.p1 * r) / r;
    if (EV) v = e - P.shift;
    return e * (1.0 + P.p1 * r) / r2;
  } else {   // EVAL_GAUSS
    const double e = exp(-P.p1 * r2);
    if (EV) v = P.p0 * e - P.shift;
    return P.p2 * e;
  }
}

// two neighbours (a, b) of particle i in packed FP32x2 arithmetic; masks ok_a/ok_b
// drop empty slots (they hold the particle itself: r = 0)
template <int EVAL, bool EV>
__device__ __forceinline__ void pair2(const int4& qi, const int4& qa, const int4& qb, bool ok_a,
                                      bool ok_b, const float2 sc0, const float2 sc1,
                                      const float2 sc2, const PairF& Pa, const PairF& Pb,
                                      float2& fx, float2& fy, float2& fz, float2& e, float2* w) {
  float2 dx = make_float2((float)min_image_fixed(qi.x, qa.x), (float)min_image_fixed(qi.x, qb.x));
  float2 dy = make_float2((float)min_image_fixed(qi.y, qa.y), (float)min_image_fixed(qi.y, qb.y));
  float2 dz = make_float2((float)min_image_fixed(qi.z, qa.z), (float)min_image_fixed(qi.z, qb.z));
  dx = __fmul2_rn(dx, sc0);
  dy = __fmul2_rn(dy, sc1);
  dz = __fmul2_rn(dz, sc2);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  float2 f, v;
  eval_f32x2<EVAL, EV>(r2, Pa, Pb, f, v);
  const bool in_a = ok_a && r2.x < Pa.rc2, in_b = ok_b && r2.y < Pb.rc2;
  f.x = in_a ? f.x : 0.f;   // select: an empty slot's inf/NaN never propagates
  f.y = in_b ? f.y : 0.f;
  fx = __ffma2_rn(f, dx, fx);
  fy = __ffma2_rn(f, dy, fy);
  fz = __ffma2_rn(f, dz, fz);
  if (EV) {
    v.x = in_a ? 0.5f * v.x : 0.f;
    v.y = in_b ? 0.5f * v.y : 0.f;
    e = __fadd2_rn(e, v);
    const float2 hf = __fmul2_rn(make_float2(0.5f, 0.5f), f);
    const float2 hx = __fmul2_rn(hf, dx), hy = __fmul2_rn(hf, dy), hz = __fmul2_rn(hf, dz);
    w[0] = __ffma2_rn(hx, dx, w[0]);
    w[1] = __ffma2_rn(hx, dy, w[1]);
    w[2] = __ffma2_rn(hx, dz, w[2]);
    w[3] = __ffma2_rn(hy, dy, w[3]);
    w[4] = __ffma2_rn(hy, dz, w[4]);
    w[5] = __ffma2_rn(hz, dz, w[5]);
  }
}

// MODE_FORCE: forces at the current positions (readouts); MODE_EV: also the
// energy / virial / v.v partial sums; MODE_STEP: the step kernel -- forces, then each
// particle's velocity Verlet update into the next shadow buffer (step_core.cuh), then
// the end-of-step decisions by the last of `total_blocks` blocks.  A system that is
// frozen (device error) or at its step limit is skipped in step mode.
template <int PREC, int TPP, int MT, int MODE, int EVAL>
__device__ __forceinline__ void force_body(const SysDev* __restrict__ sysv,
                                           const Tile* __restrict__ tiles, GroupCtl* ctl,
                                           int nsys, int total_blocks,
                                           cudaGraphConditionalHandle cond, int use_cond) {
  constexpr bool EV = MODE == MODE_EV, STEP = MODE == MODE_STEP, NVTA = MODE == MODE_NVT_A;
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  if (threadIdx.x == 0 && t.first == 0) atomicAdd(&s.flags->launches, 1ull);
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
  const FlagWords fw = load_flag_words(s.flags);
  const longlong2 sl = load_flag_pair(&s.flags->step);   // (step, step_limit)
  const bool active = !(STEP || NVTA) || (fw.error == 0 && (sl.y < 0 || sl.x < sl.y));   // uniform
  const long long step = sl.x;
  bool need = false, bad = false;
  double uu = 0.0;   // NVT: v.v after the closing half
  const int nt = s.ntypes;
  constexpr bool SMEM_TAB = PREC == GBMD_MIXED ? MT == 2 : MT != 0;
  __shared__ PairF tabf[SMEM_TAB ? MAXT2 : 1];
  __shared__ PairD tabd[SMEM_TAB ? MAXT2 : 1];
  if (SMEM_TAB) {
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) {
      if (PREC == GBMD_MIXED) {
        tabf[k] = s.pf[k];
      } else {   // FP64: the FP32 cut for the pre-test, and the FP64 coefficients
        tabf[k] = s.pf[k];
        tabd[k] = s.pd[k];
      }
    }
    __syncthreads();
  }
  const int g = threadIdx.x / TPP, h = threadIdx.x % TPP;
  const bool valid = g < t.count;
  const int i = t.first + (valid ? g : 0);
  if (active) {
  const int n = valid ? s.nn[i] : 0;
  if (STEP && valid && h == 0) prefetch_particle(s, i);   // in flight during the gathers
  const int groups = (n + 3) >> 2;
  const int4* __restrict__ nl4 = reinterpret_cast<const int4*>(s.nl) + i;
  const size_t stride = (size_t)s.nl_stride;
  const int cap_groups = s.cap >> 2;
  // first slot group of this lane, fetched before the count is known
  int4 jn = h < cap_groups ? __ldg(nl4 + (size_t)h * stride) : make_int4(i, i, i, i);

  if (PREC == GBMD_MIXED) {
    const int4* __restrict__ qv = q_at(s, step);
    const int4 qi = qv[i];
    const float2 sc0 = make_float2(s.fscale[0], s.fscale[0]);
    const float2 sc1 = make_float2(s.fscale[1], s.fscale[1]);
    const float2 sc2 = make_float2(s.fscale[2], s.fscale[2]);
    const PairF p0 = s.pf[0];
    // two types: particle i's row of the pair table stays in registers, so a
    // neighbour's parameters are a select, not a shared-memory load per pair
    const PairF r0 = MT == 1 ? s.pf[qi.w * nt] : p0;
    const PairF r1 = MT == 1 ? s.pf[qi.w * nt + nt - 1] : p0;
    auto par = [&](int tj) -> PairF {
      if (MT == 0) return p0;
      if (MT == 1) return tj ? r1 : r0;
      return tabf[qi.w * nt + tj];
    };
    float2 fx = make_float2(0.f, 0.f), fy = fx, fz = fx, e = fx;
    float2 w[6] = {fx, fx, fx, fx, fx, fx};
    for (int gg = h; gg < groups; gg += TPP) {
      const int4 jc = jn;
      if (gg + TPP < groups) jn = __ldg(nl4 + (size_t)(gg + TPP) * stride);
      const int k0 = gg << 2;
      const bool o0 = k0 < n, o1 = k0 + 1 < n, o2 = k0 + 2 < n, o3 = k0 + 3 < n;
      const int4 q0 = __ldg(qv + (o0 ? jc.x : i));
      const int4 q1 = __ldg(qv + (o1 ? jc.y : i));
      const int4 q2 = __ldg(qv + (o2 ? jc.z : i));
      const int4 q3 = __ldg(qv + (o3 ? jc.w : i));
      const PairF P0 = par(q0.w), P1 = par(q1.w), P2 = par(q2.w), P3 = par(q3.w);
      pair2<EVAL, EV>(qi, q0, q1, o0, o1, sc0, sc1, sc2, P0, P1, fx, fy, fz, e, w);
      pair2<EVAL, EV>(qi, q2, q3, o2, o3, sc0, sc1, sc2, P2, P3, fx, fy, fz, e, w);
    }
    // the two halves of each packed accumulator, then the TPP lanes
    const float Fx = group_sum<TPP>(fx.x + fx.y);
    const float Fy = group_sum<TPP>(fy.x + fy.y);
    const float Fz = group_sum<TPP>(fz.x + fz.y);
    float E = 0.f, W[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (EV) {
      E = group_sum<TPP>(e.x + e.y);
      for (int c = 0; c < 6; ++c) W[c] = group_sum<TPP>(w[c].x + w[c].y);
    }
    if (STEP) {   // the step needs no stored force: each lane-0 integrates its particle
      if (valid && h == 0) {
        const double f[3] = {widen_f32(Fx, bad), widen_f32(Fy, bad), widen_f32(Fz, bad)};
        integrate_one<PREC>(s, i, qi.w, f, fw.v_full, load_particle(s, i), q_at(s, step + 1), nullptr,
                            need, bad);
      }
    } else if (NVTA) {   // closing half kick and scaling; the second half reads F
      if (valid && h == 0) {
        const double f[3] = {widen_f32(Fx, bad), widen_f32(Fy, bad), widen_f32(Fz, bad)};
        uu = nvt_close(s, i, f, fw.v_full);
        s.f32[i] = make_float4(Fx, Fy, Fz, 0.f);
      }
    } else if (valid && h == 0) {
      s.f32[i] = make_float4(Fx, Fy, Fz, EV ? E : 0.f);
    }
    if (EV) {
      double vals[NPART] = {valid ? (double)E : 0.0};
      for (int c = 0; c < 6; ++c) vals[c + 1] = valid ? (double)W[c] : 0.0;
      vals[7] = valid ? vsq(s, i, Fx, Fy, Fz, fw.v_full) : 0.0;
      if (valid && h == 0 && s.pp_u) {
        s.pp_u[i] = vals[0];
        for (int c = 0; c < 6; ++c) s.pp_w[6 * (size_t)i + c] = vals[c + 1];
      }
      reduce_partials<TPP, 512>(vals, s.partials + 8 * (size_t)blockIdx.x);
    }
  } else {
    const double4_32a* __restrict__ pv = p64_at(s, step);
    const double4_32a pi = pv[i];
    const int ti = (int)__double_as_longlong(pi.w);
    // the FP32 pre-test reads the fixed-point shadow of the same positions
    const int4* __restrict__ qv = q_at(s, step);
    const int4 qi = qv[i];
    const float fs0 = s.fscale[0], fs1 = s.fscale[1], fs2 = s.fscale[2];
    const float cut0 = s.pf[0].rc2 * FP64_PRETEST_MARGIN;
    const double L0 = s.L[0], L1 = s.L[1], L2 = s.L[2];
    const int h0 = __double2hiint(s.halfL[0]), h1 = __double2hiint(s.halfL[1]),
              h2 = __double2hiint(s.halfL[2]);
    const PairD p0 = s.pd[0];
    double fx = 0, fy = 0, fz = 0, e = 0;
    double w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    for (int gg = h; gg < groups; gg += TPP) {
      const int4 jc = jn;
      if (gg + TPP < groups) jn = __ldg(nl4 + (size_t)(gg + TPP) * stride);
      const int k0 = gg << 2;
      const int jj[4] = {jc.x, jc.y, jc.z, jc.w};
      double4_32a pp[4];
      int4 qq[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = k0 + u < n ? jj[u] : i;   // own slot: unused
        pp[u] = pv[j];
        qq[u] = __ldg(qv + j);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        // FP32 pre-test on the fixed-point difference (the exact minimum image): a
        // pair beyond r_cut by more than the margin skips the FP64 work, which it
        // would not pass; every other pair is decided in FP64 below
        const float ex = (float)min_image_fixed(qi.x, qq[u].x) * fs0;
        const float ey = (float)min_image_fixed(qi.y, qq[u].y) * fs1;
        const float ez = (float)min_image_fixed(qi.z, qq[u].z) * fs2;
        const float r2f = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        const float cut = MT ? tabf[ti * nt + qq[u].w].rc2 * FP64_PRETEST_MARGIN : cut0;
        if (!(k0 + u < n) || !(r2f < cut)) continue;
        const double4_32a pj = pp[u];
        double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        // minimum image: |d| < L; the test on the high words is exact except within
        // 2^-20 of L/2, where either choice leaves |d| ~ L/2 > r_cut.  Only pairs
        // across a box face need it, so a warp takes the correction (FP64 adds on
        // every lane once the compiler turns it into selects) only when one of its
        // pairs does
        const bool wx = (__double2hiint(dx) & 0x7fffffff) > h0;
        const bool wy = (__double2hiint(dy) & 0x7fffffff) > h1;
        const bool wz = (__double2hiint(dz) & 0x7fffffff) > h2;
        if (__any_sync(__activemask(), wx || wy || wz)) {
          if (wx) dx -= copysign(L0, dx);
          if (wy) dy -= copysign(L1, dy);
          if (wz) dz -= copysign(L2, dz);
        }
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const PairD P = MT ? tabd[ti * nt + (int)__double_as_longlong(pj.w)] : p0;
        // both positive, so the bit patterns order like the values
        const bool in = k0 + u < n && __double_as_longlong(r2) < __double_as_longlong(P.rc2);
        if (in) {
          double v;
          const double f = eval_f64<EVAL, EV>(r2, P, v);
          fx = fma(f, dx, fx);
          fy = fma(f, dy, fy);
          fz = fma(f, dz, fz);
          if (EV) {
            e += 0.5 * v;
            const double hf = 0.5 * f;
            w0 = fma(hf * dx, dx, w0);
            w1 = fma(hf * dx, dy, w1);
            w2 = fma(hf * dx, dz, w2);
            w3 = fma(hf * dy, dy, w3);
            w4 = fma(hf * dy, dz, w4);
            w5 = fma(hf * dz, dz, w5);
          }
        }
      }
    }
    fx = group_sum<TPP>(fx);
    fy = group_sum<TPP>(fy);
    fz = group_sum<TPP>(fz);
    if (EV) {
      e = group_sum<TPP>(e);
      w0 = group_sum<TPP>(w0); w1 = group_sum<TPP>(w1); w2 = group_sum<TPP>(w2);
      w3 = group_sum<TPP>(w3); w4 = group_sum<TPP>(w4); w5 = group_sum<TPP>(w5);
    }
    if (STEP) {
      if (valid && h == 0) {
        const double f[3] = {fx, fy, fz};
        bad |= !isfinite(fx) || !isfinite(fy) || !isfinite(fz);
        integrate_one<PREC>(s, i, ti, f, fw.v_full, load_particle(s, i), q_at(s, step + 1),
                            p64_at(s, step + 1), need, bad);
      }
    } else if (NVTA) {
      if (valid && h == 0) {
        const double f[3] = {fx, fy, fz};
        uu = nvt_close(s, i, f, fw.v_full);
        s.f64[i] = make_double4_32a(fx, fy, fz, 0.0);
      }
    } else if (valid && h == 0) {
      s.f64[i] = make_double4_32a(fx, fy, fz, EV ? e : 0.0);
    }
    if (EV) {
      double vals[NPART] = {valid ? e : 0.0,  valid ? w0 : 0.0, valid ? w1 : 0.0, valid ? w2 : 0.0,
                            valid ? w3 : 0.0, valid ? w4 : 0.0, valid ? w5 : 0.0,
                            valid ? vsq(s, i, fx, fy, fz, fw.v_full) : 0.0};
      if (valid && h == 0 && s.pp_u) {
        s.pp_u[i] = vals[0];
        for (int c = 0; c < 6; ++c) s.pp_w[6 * (size_t)i + c] = vals[c + 1];
      }
      reduce_partials<TPP, 512>(vals, s.partials + 8 * (size_t)blockIdx.x);
    }
  }
  }   // active
  if (STEP) step_tail(s, sysv, ctl, nsys, total_blocks, cond, use_cond, need, bad);
  if (NVTA) {
    if (bad) atomicCAS(&s.flags->error, 0, (int)DEV_NONFINITE);
    nvt_half_tail(s, sysv, ctl, nsys, total_blocks, uu);
  }
}


template <int PREC, int TPP, int MT, int MODE, int EVAL>
__global__ void __launch_bounds__(512) k_force(const SysDev* __restrict__ sysv,
                                               const Tile* __restrict__ tiles, GroupCtl* ctl,
                                               int nsys, int total_blocks,
                                               cudaGraphConditionalHandle cond, int use_cond) {
  force_body<PREC, TPP, MT, MODE, EVAL>(sysv, tiles, ctl, nsys, total_blocks, cond, use_cond);
}

// The mixed-precision step kernel with one lane per particle (the large systems)
// under a register cap: fewer registers let more warps keep gathers in flight.  56
// measured 5% faster than the 64 the compiler picks on the Kob-Andersen 10^6 step
// (199 against 209 us); 48 and 40 spill and run slower.  With two lanes per particle
// (the 64k fluid) the same cap made the step 8% slower, so it stays with one lane.
constexpr int STEP1_MAXREG = 56;
template <int MT, int EVAL>
__global__ void __maxnreg__(STEP1_MAXREG)
    k_force_step1(const SysDev* __restrict__ sysv, const Tile* __restrict__ tiles, GroupCtl* ctl,
                  int nsys, int total_blocks, cudaGraphConditionalHandle cond, int use_cond) {
  force_body<GBMD_MIXED, 1, MT, MODE_STEP, EVAL>(sysv, tiles, ctl, nsys, total_blocks, cond,
                                                 use_cond);
}

// the k_force variant for (precision, threads per particle, table mode, mode) with
// evaluator EVAL; only LJ has the two-type register table (mode 1)
template <int EVAL, int PREC, int TPP, int MT>
void* k_force_mode(int mode) {
  switch (mode) {
    case MODE_EV: return (void*)k_force<PREC, TPP, MT, MODE_EV, EVAL>;
    case MODE_STEP:
      if constexpr (PREC == GBMD_MIXED && TPP == 1) return (void*)k_force_step1<MT, EVAL>;
      else return (void*)k_force<PREC, TPP, MT, MODE_STEP, EVAL>;
    case MODE_NVT_A: return (void*)k_force<PREC, TPP, MT, MODE_NVT_A, EVAL>;
    default: return (void*)k_force<PREC, TPP, MT, MODE_FORCE, EVAL>;
  }
}

template <int EVAL, int PREC, int TPP>
void* k_force_table(int mt, int mode) {
  if constexpr (PREC == GBMD_FP64 || EVAL != EVAL_LJ) {
    return mt ? k_force_mode<EVAL, PREC, TPP, 2>(mode) : k_force_mode<EVAL, PREC, TPP, 0>(mode);
  } else {
    if (mt == 1) return k_force_mode<EVAL, PREC, TPP, 1>(mode);
    if (mt == 2) return k_force_mode<EVAL, PREC, TPP, 2>(mode);
    return k_force_mode<EVAL, PREC, TPP, 0>(mode);
  }
}

template <int EVAL, int PREC>
void* k_force_tpp(int tpp, int mt, int mode) {
  switch (tpp) {
    case 1: return k_force_table<EVAL, PREC, 1>(mt, mode);
    case 2: return k_force_table<EVAL, PREC, 2>(mt, mode);
    default: return k_force_table<EVAL, PREC, 4>(mt, mode);
  }
}

// every k_force variant of evaluator EVAL (instantiated in its own translation unit)
template <int EVAL>
void* k_force_variant(int prec, int tpp, int mt, int mode) {
  return prec == GBMD_FP64 ? k_force_tpp<EVAL, GBMD_FP64>(tpp, mt, mode)
                           : k_force_tpp<EVAL, GBMD_MIXED>(tpp, mt, mode);
}
void* k_force_variant_mie(int prec, int tpp, int mt, int mode);      // k_force_mie.cu
void* k_force_variant_yukawa(int prec, int tpp, int mt, int mode);   // k_force_yukawa.cu
void* k_force_variant_gauss(int prec, int tpp, int mt, int mode);    // k_force_gauss.cu

}  // namespace gbmd
