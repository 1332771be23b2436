// k_force.cu -- the LJ (and WCA) instances of the pair-force gather (k_force.cuh),
// the second half of the NVT step, the staged LJ force path, and the launch builders
// of every force kernel.
#include <mutex>
#include <set>
#include <utility>

#include "k_force.cuh"

namespace gbmd {

KernelCall make_call(void* f, int grid, int block, size_t smem);

template <typename T>
static void put(KernelCall& k, const T& v) {
  static_assert(sizeof(T) <= 16, "arg too large");
  memcpy(k.store[k.nargs], &v, sizeof(T));
  ++k.nargs;
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
        pair2<EVAL_LJ, EV>(qi, qa, qb, ka < n, kb < n, sc0, sc1, sc2, par(qa.w), par(qb.w), fx,
                           fy, fz, e, w);
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

// multi: 0 = one type, 1 = at most two types, 2 = up to MAXT types
KernelCall force_call(int prec, int multi, int mode, int tpp, int block, const SysDev* d,
                      const Tile* tiles_f, int ntiles, GroupCtl* ctl, const StepArgs& sa,
                      int eval) {
  // the FP64 kernel is FP64-pipe bound: its table stays in shared memory
  void* f;
  switch (eval) {
    case EVAL_MIE: f = k_force_variant_mie(prec, tpp, multi, mode); break;
    case EVAL_YUKAWA: f = k_force_variant_yukawa(prec, tpp, multi, mode); break;
    case EVAL_GAUSS: f = k_force_variant_gauss(prec, tpp, multi, mode); break;
    default: f = k_force_variant<EVAL_LJ>(prec, tpp, multi, mode);
  }
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
