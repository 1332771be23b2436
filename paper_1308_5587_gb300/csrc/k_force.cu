// k_force.cu -- LJ pair-force gather over the full Verlet neighbour list (K5).
//
// Section 3.1 / Listing 1: md.pair.lj(r_cut) with per type-pair epsilon, sigma;
// Section 5 names the GPU technique: several threads per particle with warp-level
// reductions.  The paper gives no formula; the kernel computes, for every listed
// neighbour j of particle i with r^2 < r_cut,ij^2 (strict):
//   F_i += f d_ij,  f = 24 eps [2 (sigma/r)^12 - (sigma/r)^6] / r^2,  d_ij = x_i - x_j,
// and optionally u_i += 1/2 (4 eps [(sigma/r)^12 - (sigma/r)^6] - V_LJ(r_cut)) and
// W_i,ab += 1/2 d_a f d_b, whose per-tile sums are reduced in FP64.
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
// arithmetic runs two neighbours at a time in packed FP32x2 operations; per-particle
// sums are FP32.
// FP64: positions come from the double4 shadow p64; the minimum image is one
// conditional correction by L (|d| < L for wrapped coordinates); all arithmetic FP64.
#include "launch.cuh"

namespace gbmd {

KernelCall make_call(void* f, int grid, int block, size_t smem);

template <typename T>
static void put(KernelCall& k, const T& v) {
  static_assert(sizeof(T) <= 16, "arg too large");
  memcpy(k.store[k.nargs], &v, sizeof(T));
  ++k.nargs;
}

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

// FP64 block reduction of 7 per-particle values into partials[tile][0..6] (fixed order)
template <int TPP, int BLOCK_MAX>
__device__ void reduce_partials(const double* vals, double* out) {
  constexpr int GMAX = BLOCK_MAX / TPP;
  __shared__ double sh[7][GMAX];
  const int g = threadIdx.x / TPP, l = threadIdx.x % TPP;
  const int ng = blockDim.x / TPP;
  if (l == 0)
    for (int c = 0; c < 7; ++c) sh[c][g] = vals[c];
  __syncthreads();
  if (threadIdx.x < 7) {
    double acc = 0;
    for (int k = 0; k < ng; ++k) acc += sh[threadIdx.x][k];
    out[threadIdx.x] = acc;
  }
}

// two neighbours (a, b) of particle i in packed FP32x2 arithmetic; masks ok_a/ok_b
// drop empty slots (they hold the particle itself: r = 0)
template <bool EV>
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
  const float2 r2i = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
  const float2 r6i = __fmul2_rn(__fmul2_rn(r2i, r2i), r2i);
  const float2 lj1 = make_float2(Pa.lj1, Pb.lj1), mlj2 = make_float2(-Pa.lj2, -Pb.lj2);
  float2 f = __fmul2_rn(__fmul2_rn(r2i, r6i), __ffma2_rn(lj1, r6i, mlj2));
  const bool in_a = ok_a && r2.x < Pa.rc2, in_b = ok_b && r2.y < Pb.rc2;
  f.x = in_a ? f.x : 0.f;   // select: an empty slot's inf/NaN never propagates
  f.y = in_b ? f.y : 0.f;
  fx = __ffma2_rn(f, dx, fx);
  fy = __ffma2_rn(f, dy, fy);
  fz = __ffma2_rn(f, dz, fz);
  if (EV) {
    const float2 c12 = make_float2(Pa.c12, Pb.c12), mc6 = make_float2(-Pa.c6, -Pb.c6);
    const float2 msh = make_float2(-Pa.shift, -Pb.shift);
    float2 v = __ffma2_rn(r6i, __ffma2_rn(c12, r6i, mc6), msh);
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

template <int PREC, int TPP, bool MULTI, bool EV>
__global__ void __launch_bounds__(512) k_force(const SysDev* __restrict__ sysv,
                                               const Tile* __restrict__ tiles, GroupCtl* ctl,
                                               int force_all) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  if (threadIdx.x == 0 && t.first == 0) atomicAdd(&s.flags->launches, 1ull);
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
  if (!force_all) {
    const volatile Flags* vf = s.flags;
    if (!vf->active || vf->error) return;   // uniform over the block
  }
  const int nt = s.ntypes;
  __shared__ PairF tabf[MULTI ? MAXT2 : 1];
  __shared__ PairD tabd[MULTI ? MAXT2 : 1];
  if (MULTI) {
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) {
      if (PREC == GBMD_MIXED) tabf[k] = s.pf[k]; else tabd[k] = s.pd[k];
    }
    __syncthreads();
  }
  const int g = threadIdx.x / TPP, h = threadIdx.x % TPP;
  const bool valid = g < t.count;
  const int i = t.first + (valid ? g : 0);
  const int n = valid ? s.nn[i] : 0;
  const int groups = (n + 3) >> 2;
  const int4* __restrict__ nl4 = reinterpret_cast<const int4*>(s.nl) + i;
  const size_t stride = (size_t)s.nl_stride;
  const int cap_groups = s.cap >> 2;
  // first slot group of this lane, fetched before the count is known
  int4 jn = h < cap_groups ? __ldg(nl4 + (size_t)h * stride) : make_int4(i, i, i, i);

  if (PREC == GBMD_MIXED) {
    const int4 qi = s.q[i];
    const float2 sc0 = make_float2(s.fscale[0], s.fscale[0]);
    const float2 sc1 = make_float2(s.fscale[1], s.fscale[1]);
    const float2 sc2 = make_float2(s.fscale[2], s.fscale[2]);
    const PairF p0 = s.pf[0];
    const int4* __restrict__ qv = s.q;
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
      const PairF P0 = MULTI ? tabf[qi.w * nt + q0.w] : p0;
      const PairF P1 = MULTI ? tabf[qi.w * nt + q1.w] : p0;
      const PairF P2 = MULTI ? tabf[qi.w * nt + q2.w] : p0;
      const PairF P3 = MULTI ? tabf[qi.w * nt + q3.w] : p0;
      pair2<EV>(qi, q0, q1, o0, o1, sc0, sc1, sc2, P0, P1, fx, fy, fz, e, w);
      pair2<EV>(qi, q2, q3, o2, o3, sc0, sc1, sc2, P2, P3, fx, fy, fz, e, w);
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
    if (valid && h == 0) s.f32[i] = make_float4(Fx, Fy, Fz, EV ? E : 0.f);
    if (EV) {
      double vals[7] = {valid ? (double)E : 0.0};
      for (int c = 0; c < 6; ++c) vals[c + 1] = valid ? (double)W[c] : 0.0;
      if (valid && h == 0 && s.pp_u) {
        s.pp_u[i] = vals[0];
        for (int c = 0; c < 6; ++c) s.pp_w[6 * (size_t)i + c] = vals[c + 1];
      }
      reduce_partials<TPP, 512>(vals, s.partials + 8 * (size_t)blockIdx.x);
    }
  } else {
    const double4_32a pi = s.p64[i];
    const int ti = (int)__double_as_longlong(pi.w);
    const double L0 = s.L[0], L1 = s.L[1], L2 = s.L[2];
    const int h0 = __double2hiint(s.halfL[0]), h1 = __double2hiint(s.halfL[1]),
              h2 = __double2hiint(s.halfL[2]);
    const PairD p0 = s.pd[0];
    const double4_32a* __restrict__ pv = s.p64;
    double fx = 0, fy = 0, fz = 0, e = 0;
    double w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    for (int gg = h; gg < groups; gg += TPP) {
      const int4 jc = jn;
      if (gg + TPP < groups) jn = __ldg(nl4 + (size_t)(gg + TPP) * stride);
      const int k0 = gg << 2;
      const int jj[4] = {jc.x, jc.y, jc.z, jc.w};
      double4_32a pp[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) pp[u] = pv[k0 + u < n ? jj[u] : i];   // own slot: unused
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double4_32a pj = pp[u];
        double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        // minimum image: |d| < L; the test on the high words is exact except within
        // 2^-20 of L/2, where either choice leaves |d| ~ L/2 > r_cut
        if ((__double2hiint(dx) & 0x7fffffff) > h0) dx -= copysign(L0, dx);
        if ((__double2hiint(dy) & 0x7fffffff) > h1) dy -= copysign(L1, dy);
        if ((__double2hiint(dz) & 0x7fffffff) > h2) dz -= copysign(L2, dz);
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const PairD P = MULTI ? tabd[ti * nt + (int)__double_as_longlong(pj.w)] : p0;
        // both positive, so the bit patterns order like the values
        const bool in = k0 + u < n && __double_as_longlong(r2) < __double_as_longlong(P.rc2);
        if (in) {
          const double r2i = __drcp_rn(r2);
          const double r6i = r2i * r2i * r2i;
          const double f = r2i * r6i * fma(P.lj1, r6i, -P.lj2);
          fx = fma(f, dx, fx);
          fy = fma(f, dy, fy);
          fz = fma(f, dz, fz);
          if (EV) {
            e += 0.5 * fma(r6i, fma(P.c12, r6i, -P.c6), -P.shift);
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
    if (valid && h == 0) s.f64[i] = make_double4_32a(fx, fy, fz, EV ? e : 0.0);
    if (EV) {
      double vals[7] = {valid ? e : 0.0,  valid ? w0 : 0.0, valid ? w1 : 0.0, valid ? w2 : 0.0,
                        valid ? w3 : 0.0, valid ? w4 : 0.0, valid ? w5 : 0.0};
      if (valid && h == 0 && s.pp_u) {
        s.pp_u[i] = vals[0];
        for (int c = 0; c < 6; ++c) s.pp_w[6 * (size_t)i + c] = vals[c + 1];
      }
      reduce_partials<TPP, 512>(vals, s.partials + 8 * (size_t)blockIdx.x);
    }
  }
}

bool tpp_supported(int tpp) { return tpp == 1 || tpp == 2 || tpp == 4; }

template <int PREC, int TPP>
static void* pick3(int multi, int ev) {
  if (multi) return ev ? (void*)k_force<PREC, TPP, true, true> : (void*)k_force<PREC, TPP, true, false>;
  return ev ? (void*)k_force<PREC, TPP, false, true> : (void*)k_force<PREC, TPP, false, false>;
}

template <int PREC>
static void* pick2(int tpp, int multi, int ev) {
  switch (tpp) {
    case 1: return pick3<PREC, 1>(multi, ev);
    case 2: return pick3<PREC, 2>(multi, ev);
    default: return pick3<PREC, 4>(multi, ev);
  }
}

KernelCall force_call(int prec, int multi, int ev, int tpp, int block, const SysDev* d,
                      const Tile* tiles_f, int ntiles, GroupCtl* ctl, int force_all) {
  void* f = prec == GBMD_FP64 ? pick2<GBMD_FP64>(tpp, multi, ev) : pick2<GBMD_MIXED>(tpp, multi, ev);
  KernelCall k = make_call(f, ntiles, block, 0);
  put(k, d); put(k, tiles_f); put(k, ctl); put(k, force_all);
  return k;
}

}  // namespace gbmd
