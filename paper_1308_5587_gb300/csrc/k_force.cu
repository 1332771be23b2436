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
// Mapping: TPP lanes cooperate on one particle; lane l takes the row entries
// l, l+TPP, ... (consecutive lanes read consecutive 4-byte indices, so a group
// reads whole 32-byte sectors of its row), then the TPP partial sums are combined
// with xor shuffles in a fixed order (deterministic).
//
// MIXED: positions come from the 32-bit fixed-point shadow q (int4: x, y, z, type).
// The int32 difference of two fixed-point coordinates is the minimum-image
// displacement exactly; it is converted to FP32 and scaled by L/2^32.  All pair
// arithmetic and the per-particle sums are FP32.
// FP64: positions come from the double4_32a shadow p64; the minimum image is one
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

// FP64 block reduction of 7 per-group values into partials[tile][0..6] (fixed order)
template <int TPP, int BLOCK_MAX>
__device__ void reduce_partials(double* vals, double* out) {
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

template <int PREC, int TPP, bool MULTI, bool EV>
__global__ void __launch_bounds__(1024) k_force(const SysDev* __restrict__ sysv,
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
  const int g = threadIdx.x / TPP, l = threadIdx.x % TPP;
  const bool valid = g < t.count;
  const int i = t.first + (valid ? g : 0);
  const int n = valid ? s.nn[i] : 0;
  const int* __restrict__ row = s.nl + (size_t)i * s.cap;

  if (PREC == GBMD_MIXED) {
    const int4 qi = s.q[i];
    const float fs0 = s.fscale[0], fs1 = s.fscale[1], fs2 = s.fscale[2];
    const PairF p0 = s.pf[0];
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    float w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f;
#pragma unroll 4
    for (int k = l; k < n; k += TPP) {
      const int j = __ldg(row + k);
      const int4 qj = __ldg(s.q + j);
      const float dx = (float)min_image_fixed(qi.x, qj.x) * fs0;
      const float dy = (float)min_image_fixed(qi.y, qj.y) * fs1;
      const float dz = (float)min_image_fixed(qi.z, qj.z) * fs2;
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const PairF P = MULTI ? tabf[qi.w * nt + qj.w] : p0;
      const float r2i = rcp_approx(r2);
      const float r6i = r2i * r2i * r2i;
      float f = r2i * r6i * fmaf(P.lj1, r6i, -P.lj2);
      const bool in = r2 < P.rc2;
      f = in ? f : 0.f;
      fx = fmaf(f, dx, fx);
      fy = fmaf(f, dy, fy);
      fz = fmaf(f, dz, fz);
      if (EV) {
        const float v = fmaf(r6i, fmaf(P.c12, r6i, -P.c6), -P.shift);
        e += in ? 0.5f * v : 0.f;
        const float hf = 0.5f * f;
        w0 = fmaf(hf * dx, dx, w0);
        w1 = fmaf(hf * dx, dy, w1);
        w2 = fmaf(hf * dx, dz, w2);
        w3 = fmaf(hf * dy, dy, w3);
        w4 = fmaf(hf * dy, dz, w4);
        w5 = fmaf(hf * dz, dz, w5);
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
    if (valid && l == 0) s.f32[i] = make_float4(fx, fy, fz, EV ? e : 0.f);
    if (EV) {
      double vals[7] = {valid ? (double)e : 0.0, valid ? (double)w0 : 0.0,
                        valid ? (double)w1 : 0.0, valid ? (double)w2 : 0.0,
                        valid ? (double)w3 : 0.0, valid ? (double)w4 : 0.0,
                        valid ? (double)w5 : 0.0};
      if (valid && l == 0 && s.pp_u) {
        s.pp_u[i] = vals[0];
        for (int c = 0; c < 6; ++c) s.pp_w[6 * (size_t)i + c] = vals[c + 1];
      }
      reduce_partials<TPP, 1024>(vals, s.partials + 8 * (size_t)blockIdx.x);
    }
  } else {
    const double4_32a pi = s.p64[i];
    const int ti = (int)__double_as_longlong(pi.w);
    const double L0 = s.L[0], L1 = s.L[1], L2 = s.L[2];
    const int h0 = __double2hiint(s.halfL[0]), h1 = __double2hiint(s.halfL[1]),
              h2 = __double2hiint(s.halfL[2]);
    const PairD p0 = s.pd[0];
    double fx = 0, fy = 0, fz = 0, e = 0;
    double w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
#pragma unroll 2
    for (int k = l; k < n; k += TPP) {
      const int j = __ldg(row + k);
      const double4_32a pj = s.p64[j];
      double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
      // minimum image: |d| < L; the test on the high words is exact except within
      // 2^-20 of L/2, where either choice leaves |d| ~ L/2 > r_cut
      if ((__double2hiint(dx) & 0x7fffffff) > h0) dx -= copysign(L0, dx);
      if ((__double2hiint(dy) & 0x7fffffff) > h1) dy -= copysign(L1, dy);
      if ((__double2hiint(dz) & 0x7fffffff) > h2) dz -= copysign(L2, dz);
      const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
      const PairD P = MULTI ? tabd[ti * nt + (int)__double_as_longlong(pj.w)] : p0;
      const bool in = __double_as_longlong(r2) < __double_as_longlong(P.rc2);  // both > 0
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
    fx = group_sum<TPP>(fx);
    fy = group_sum<TPP>(fy);
    fz = group_sum<TPP>(fz);
    if (EV) {
      e = group_sum<TPP>(e);
      w0 = group_sum<TPP>(w0); w1 = group_sum<TPP>(w1); w2 = group_sum<TPP>(w2);
      w3 = group_sum<TPP>(w3); w4 = group_sum<TPP>(w4); w5 = group_sum<TPP>(w5);
    }
    if (valid && l == 0) s.f64[i] = make_double4_32a(fx, fy, fz, EV ? e : 0.0);
    if (EV) {
      double vals[7] = {valid ? e : 0.0,  valid ? w0 : 0.0, valid ? w1 : 0.0, valid ? w2 : 0.0,
                        valid ? w3 : 0.0, valid ? w4 : 0.0, valid ? w5 : 0.0};
      if (valid && l == 0 && s.pp_u) {
        s.pp_u[i] = vals[0];
        for (int c = 0; c < 6; ++c) s.pp_w[6 * (size_t)i + c] = vals[c + 1];
      }
      reduce_partials<TPP, 1024>(vals, s.partials + 8 * (size_t)blockIdx.x);
    }
  }
}

bool tpp_supported(int tpp) { return tpp == 4 || tpp == 8 || tpp == 16 || tpp == 32; }

template <int PREC, int TPP>
static void* pick3(int multi, int ev) {
  if (multi) return ev ? (void*)k_force<PREC, TPP, true, true> : (void*)k_force<PREC, TPP, true, false>;
  return ev ? (void*)k_force<PREC, TPP, false, true> : (void*)k_force<PREC, TPP, false, false>;
}

template <int PREC>
static void* pick2(int tpp, int multi, int ev) {
  switch (tpp) {
    case 4: return pick3<PREC, 4>(multi, ev);
    case 8: return pick3<PREC, 8>(multi, ev);
    case 16: return pick3<PREC, 16>(multi, ev);
    default: return pick3<PREC, 32>(multi, ev);
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
