// k_force.cu -- LJ pair-force gather over the full Verlet neighbour list (K5).
//
// Section 3.1 / Listing 1: md.pair.lj(r_cut) with per type-pair epsilon, sigma;
// Section 5 names the GPU technique: several threads per particle with warp-level
// reductions.  The paper gives no formula; the kernel computes, for every listed
// neighbour j of particle i with r^2 < r_cut,ij^2 (strict):
//   F_i += f d_ij,  f = 24 eps [2 (sigma/r)^12 - (sigma/r)^6] / r^2,  d_ij = x_i - x_j,
// and optionally u_i += 1/2 (4 eps [(sigma/r)^12 - (sigma/r)^6] - V_LJ(r_cut)) and
// W_i,ab += 1/2 d_a f d_b, whose per-tile sums are reduced in FP64 together with the
// sum of v_i . v_i (kinetic energy, from the full-step velocity).
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
#include <mutex>
#include <set>
#include <utility>

#include "launch.cuh"
#include "step_core.cuh"

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

// MODE_FORCE: forces at the current positions (readouts); MODE_EV: also the
// energy / virial / v.v partial sums; MODE_STEP: the step kernel -- forces, then each
// particle's velocity Verlet update into the next shadow buffer (step_core.cuh), then
// the end-of-step decisions by the last of `total_blocks` blocks.  A system that is
// frozen (device error) or at its step limit is skipped in step mode.
template <int PREC, int TPP, int MT, int MODE>
__global__ void __launch_bounds__(512) k_force(const SysDev* __restrict__ sysv,
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
      if (PREC == GBMD_MIXED) tabf[k] = s.pf[k]; else tabd[k] = s.pd[k];
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
        const PairD P = MT ? tabd[ti * nt + (int)__double_as_longlong(pj.w)] : p0;
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

// NVT, second half of the step (one thread per particle): the opening thermostat
// scaling and half kick, drift, wrap and next shadow (integrate_one with the kick
// dt/(2m) on u exp(-xi dt/2)), then the end-of-step decisions.
template <int PREC>
__global__ void __launch_bounds__(TILE_P) k_nvt_b(const SysDev* __restrict__ sysv,
                                                  const Tile* __restrict__ tiles, GroupCtl* ctl,
                                                  int nsys, int total_blocks,
                                                  cudaGraphConditionalHandle cond, int use_cond) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  if (threadIdx.x == 0 && t.first == 0) atomicAdd(&s.flags->launches, 1ull);
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
  const FlagWords fw = load_flag_words(s.flags);
  const longlong2 sl = load_flag_pair(&s.flags->step);
  const bool active = fw.error == 0 && (sl.y < 0 || sl.x < sl.y);
  bool need = false, bad = false;
  if (active && (int)threadIdx.x < t.count) {
    const int i = t.first + threadIdx.x;
    double f[3];
    if (PREC == GBMD_FP64) {
      const double4_32a F = s.f64[i];
      f[0] = F.x; f[1] = F.y; f[2] = F.z;
    } else {
      const float4 F = s.f32[i];
      f[0] = widen_f32(F.x, bad);
      f[1] = widen_f32(F.y, bad);
      f[2] = widen_f32(F.z, bad);
    }
    ParticleState p = load_particle(s, i);
    const double so = s.nh[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) p.v[a] *= so;
    integrate_one<PREC>(s, i, s.type[i], f, 1, p, q_at(s, sl.x + 1),
                        PREC == GBMD_FP64 ? p64_at(s, sl.x + 1) : nullptr, need, bad);
  }
  step_tail(s, sysv, ctl, nsys, total_blocks, cond, use_cond, need, bad);
}

// ---- staged path: one kernel block per aligned 2x2x2 block of cells ----------------
// The block's window (the 4x4x4 cells around it, at most window_cap particles) is
// copied into shared memory as three int arrays (x, y, z with the type in z's two
// low bits): random 4-byte reads conflict far less across banks than 16-byte ones.
// Its particles' lists hold 16-bit window-local indices (ELL8: one int4 = 8 entries
// of one member), so every neighbour position comes from shared memory and the
// index stream is half as long.  One thread per particle.
template <int MT, int MODE>
__global__ void __launch_bounds__(STAGED_BLOCK) k_force_staged(const SysDev* __restrict__ sysv,
                                                               const Tile* __restrict__ tiles,
                                                               GroupCtl* ctl, int part_base,
                                                               int nsys, int total_blocks,
                                                               cudaGraphConditionalHandle cond,
                                                               int use_cond) {
  constexpr bool EV = MODE == MODE_EV, STEP = MODE == MODE_STEP;
  extern __shared__ int wsm[];   // window as three int arrays: x, y, z | type
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  if (threadIdx.x == 0 && t.first == 0) atomicAdd(&s.flags->launches, 1ull);
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
  const FlagWords fw = load_flag_words(s.flags);
  const longlong2 sl = load_flag_pair(&s.flags->step);   // (step, step_limit)
  const long long step = sl.x;
  const int b = t.first;
  const int4 info = s.blk_info[b];          // (first member, particles, window total, 0)
  // an error (e.g. a window too large) leaves nothing valid, and a window is never
  // indexed past its capacity; step mode also skips a system at its step limit
  const bool run = fw.error == 0 && info.z <= s.window_cap && (!STEP || sl.y < 0 || sl.x < sl.y);
  bool need = false, bad = false;
  if (run) {
  const int4* __restrict__ qv = q_at(s, step);
  const int* __restrict__ members = s.members;
  // stage the window: the 64 (start, offset) pairs first, then every thread copies
  // window entries tid, tid + 256, ... (independent loads, several in flight)
  __shared__ int2 wtab[WIN_CELLS];
  const int cap = s.window_cap;
  int* const wx = wsm;
  int* const wy = wsm + cap;
  int* const wz = wsm + 2 * cap;
  if (threadIdx.x < WIN_CELLS) wtab[threadIdx.x] = s.blk_win[(size_t)b * WIN_CELLS + threadIdx.x];
  __syncthreads();
  {
    constexpr int UNR = 4;
    for (int e0 = threadIdx.x; e0 < info.z; e0 += UNR * STAGED_BLOCK) {
      int src[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int e = e0 + u * STAGED_BLOCK;
        int c = 0;   // last window cell whose offset is <= e
#pragma unroll
        for (int step = 32; step > 0; step >>= 1)
          if (c + step < WIN_CELLS && wtab[c + step].y <= e) c += step;
        src[u] = e < info.z ? members[wtab[c].x + (e - wtab[c].y)] : -1;
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u)
        if (src[u] >= 0) {
          const int4 q = __ldg(qv + src[u]);
          const int e = e0 + u * STAGED_BLOCK;
          wx[e] = q.x;
          wy[e] = q.y;
          wz[e] = (q.z & ~3) | q.w;   // type in the two low bits (grid L/2^30 in z)
        }
    }
  }
  const int nt = s.ntypes;
  __shared__ PairF tabf[MT == 2 ? MAXT2 : 1];
  if (MT == 2)
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) tabf[k] = s.pf[k];
  __syncthreads();
  const float2 sc0 = make_float2(s.fscale[0], s.fscale[0]);
  const float2 sc1 = make_float2(s.fscale[1], s.fscale[1]);
  const float2 sc2 = make_float2(s.fscale[2], s.fscale[2]);
  const PairF p0 = s.pf[0];
  const size_t stride = (size_t)s.nl_stride;
  const int4* __restrict__ nl8 = reinterpret_cast<const int4*>(s.nl);
  double acc[NPART] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int vfull = fw.v_full;
  for (int pidx = threadIdx.x; pidx < info.y; pidx += STAGED_BLOCK) {
    const int m = info.x + pidx;
    const int i = members[m];
    int4 qi = qv[i];
    qi.z &= ~3;   // same z grid as the staged neighbours
    const int n = s.nn[i];
    const PairF r0 = MT == 1 ? s.pf[qi.w * nt] : p0;
    const PairF r1 = MT == 1 ? s.pf[qi.w * nt + nt - 1] : p0;
    auto par = [&](int tj) -> PairF {
      if (MT == 0) return p0;
      if (MT == 1) return tj ? r1 : r0;
      return tabf[qi.w * nt + tj];
    };
    // an empty slot (k >= n) reads window entry 0 and is masked out of the sums
    auto nb = [&](unsigned word, int k, int half) -> int4 {
      const unsigned l = k < n ? (half ? word >> 16 : word & 0xffffu) : 0u;
      const int z = wz[l];
      return make_int4(wx[l], wy[l], z & ~3, z & 3);
    };
    float2 fx = make_float2(0.f, 0.f), fy = fx, fz = fx, e = fx;
    float2 w[6] = {fx, fx, fx, fx, fx, fx};
    const int groups = (n + 7) >> 3;
    int4 nxt = groups > 0 ? __ldg(nl8 + m) : make_int4(0, 0, 0, 0);
    for (int g = 0; g < groups; ++g) {
      const int4 cur = nxt;
      if (g + 1 < groups) nxt = __ldg(nl8 + (size_t)(g + 1) * stride + m);
      const int k0 = g << 3;
      const unsigned u[4] = {(unsigned)cur.x, (unsigned)cur.y, (unsigned)cur.z, (unsigned)cur.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int ka = k0 + 2 * c, kb = ka + 1;
        const int4 qa = nb(u[c], ka, 0), qb = nb(u[c], kb, 1);
        pair2<EV>(qi, qa, qb, ka < n, kb < n, sc0, sc1, sc2, par(qa.w), par(qb.w), fx, fy, fz,
                  e, w);
      }
    }
    const float Fx = fx.x + fx.y, Fy = fy.x + fy.y, Fz = fz.x + fz.y;
    if (STEP) {
      const double f[3] = {widen_f32(Fx, bad), widen_f32(Fy, bad), widen_f32(Fz, bad)};
      integrate_one<GBMD_MIXED>(s, i, qi.w, f, vfull, load_particle(s, i), q_at(s, step + 1), nullptr,
                                need, bad);
    } else {
      s.f32[i] = make_float4(Fx, Fy, Fz, EV ? e.x + e.y : 0.f);
    }
    if (EV) {
      double v[NPART] = {(double)(e.x + e.y)};
      for (int c = 0; c < 6; ++c) v[c + 1] = (double)(w[c].x + w[c].y);
      v[7] = vsq(s, i, Fx, Fy, Fz, vfull);
      if (s.pp_u) {
        s.pp_u[i] = v[0];
        for (int c = 0; c < 6; ++c) s.pp_w[6 * (size_t)i + c] = v[c + 1];
      }
      for (int c = 0; c < NPART; ++c) acc[c] += v[c];
    }
  }
  if (EV) {   // fixed-order block reduction into this tile's partial sums
    __shared__ double red[NPART][STAGED_BLOCK];
    for (int c = 0; c < NPART; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    if (threadIdx.x < NPART) {
      double a = 0;
      for (int k = 0; k < (int)blockDim.x; ++k) a += red[threadIdx.x][k];
      s.partials[8 * (size_t)(part_base + blockIdx.x) + threadIdx.x] = a;
    }
  }
  }   // run
  if (STEP) step_tail(s, sysv, ctl, nsys, total_blocks, cond, use_cond, need, bad);
}

bool tpp_supported(int tpp) { return tpp == 1 || tpp == 2 || tpp == 4; }

template <int PREC, int TPP, int MT>
static void* pick4(int mode) {
  switch (mode) {
    case MODE_EV: return (void*)k_force<PREC, TPP, MT, MODE_EV>;
    case MODE_STEP: return (void*)k_force<PREC, TPP, MT, MODE_STEP>;
    case MODE_NVT_A: return (void*)k_force<PREC, TPP, MT, MODE_NVT_A>;
    default: return (void*)k_force<PREC, TPP, MT, MODE_FORCE>;
  }
}

template <int PREC, int TPP>
static void* pick3(int mt, int mode) {
  if constexpr (PREC == GBMD_FP64) {
    return mt ? pick4<PREC, TPP, 2>(mode) : pick4<PREC, TPP, 0>(mode);   // one FP64 table mode
  } else {
    if (mt == 1) return pick4<PREC, TPP, 1>(mode);
    if (mt == 2) return pick4<PREC, TPP, 2>(mode);
    return pick4<PREC, TPP, 0>(mode);
  }
}

template <int PREC>
static void* pick2(int tpp, int mt, int mode) {
  switch (tpp) {
    case 1: return pick3<PREC, 1>(mt, mode);
    case 2: return pick3<PREC, 2>(mt, mode);
    default: return pick3<PREC, 4>(mt, mode);
  }
}

// multi: 0 = one type, 1 = at most two types, 2 = up to MAXT types
KernelCall force_call(int prec, int multi, int mode, int tpp, int block, const SysDev* d,
                      const Tile* tiles_f, int ntiles, GroupCtl* ctl, const StepArgs& sa) {
  // the FP64 kernel is FP64-pipe bound: its table stays in shared memory
  void* f = prec == GBMD_FP64 ? pick2<GBMD_FP64>(tpp, multi, mode) : pick2<GBMD_MIXED>(tpp, multi, mode);
  KernelCall k = make_call(f, ntiles, block, 0);
  put(k, d); put(k, tiles_f); put(k, ctl); put(k, sa.nsys); put(k, sa.total_blocks);
  put(k, sa.cond); put(k, sa.use_cond);
  return k;
}

KernelCall nvt_b_call(int prec, const SysDev* d, const Tile* tiles_p, int ntiles, GroupCtl* ctl,
                      const StepArgs& sa) {
  void* f = prec == GBMD_FP64 ? (void*)k_nvt_b<GBMD_FP64> : (void*)k_nvt_b<GBMD_MIXED>;
  KernelCall k = make_call(f, ntiles, TILE_P, 0);
  put(k, d); put(k, tiles_p); put(k, ctl); put(k, sa.nsys); put(k, sa.total_blocks);
  put(k, sa.cond); put(k, sa.use_cond);
  return k;
}

KernelCall force_staged_call(int multi, int mode, const SysDev* d, const Tile* tiles_s, int ntiles,
                             GroupCtl* ctl, int part_base, int window_cap, const StepArgs& sa) {
  void* const fs[3][3] = {
      {(void*)k_force_staged<0, MODE_FORCE>, (void*)k_force_staged<0, MODE_EV>, (void*)k_force_staged<0, MODE_STEP>},
      {(void*)k_force_staged<1, MODE_FORCE>, (void*)k_force_staged<1, MODE_EV>, (void*)k_force_staged<1, MODE_STEP>},
      {(void*)k_force_staged<2, MODE_FORCE>, (void*)k_force_staged<2, MODE_EV>, (void*)k_force_staged<2, MODE_STEP>}};
  const int mt = multi < 0 ? 0 : multi > 2 ? 2 : multi;
  const int md = mode < 0 ? 0 : mode > 2 ? 2 : mode;
  void* f = fs[mt][md];
  const size_t smem = (size_t)window_cap * 3 * sizeof(int);
  {   // dynamic shared memory above the 48 KB default: once per kernel and device
    static std::mutex mu;
    static std::set<std::pair<int, void*>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (done.insert({dev, f}).second)
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  }
  KernelCall k = make_call(f, ntiles, STAGED_BLOCK, smem);
  put(k, d); put(k, tiles_s); put(k, ctl); put(k, part_base); put(k, sa.nsys);
  put(k, sa.total_blocks); put(k, sa.cond); put(k, sa.use_cond);
  return k;
}

}  // namespace gbmd
