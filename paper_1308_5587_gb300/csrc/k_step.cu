// k_step.cu -- integrate (velocity Verlet, fused leapfrog form), thermo reduction,
// and the import/export kernels of the C ABI.
//
// Velocity Verlet (NVE; Listing 1's mode_standard(dt) + run(n), NVE per Section 3.1):
//   v <- v + dt/(2m) F(t);  x <- x + dt v;  wrap;  F(t+dt);  v <- v + dt/(2m) F(t+dt).
// The closing half kick of step n and the opening half kick of step n+1 are applied
// back to back at the start of step n+1 by one kernel (k_integrate), so the stored
// velocity lags half a kick behind the full-step velocity between steps
// (Flags::v_full says when it does not, i.e. right after create / set_state).
// Positions are stored in FP64 in units of L/2^32 per axis (xq = x * 2^32 / L), so
// the drift is one FMA and the 32-bit fixed-point shadow used by the neighbour
// list and the mixed-precision force is one conversion.
#include <cstring>

#include "launch.cuh"

namespace gbmd {

// ---------------------------------------------------------------------------
// K6: kicks + drift + wrap + fixed-point shadow + displacement check, then the
// last block of the grid makes the per-step decisions for every system.
// FP64 runs at about 1/80 of the FP32 FMA rate on this part (measured: 1.6 against
// 128 FMAs per SM per clock), so the kernel keeps the FP64
// pipe to the six FMAs of the kicks and drifts plus one add per axis: the FP32
// force is widened to FP64 with integer operations (IEEE-754 field by field), and
// rint of the position uses the 1.5 * 2^52 rounding constant instead of a
// conversion instruction.
// ---------------------------------------------------------------------------

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
template <int PREC>
__global__ void __launch_bounds__(TILE_P) k_integrate(const SysDev* __restrict__ sysv,
                                                      const Tile* __restrict__ tiles,
                                                      GroupCtl* ctl, int nsys,
                                                      cudaGraphConditionalHandle cond,
                                                      int use_cond) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  Flags* fl = s.flags;
  if (threadIdx.x == 0 && t.first == 0) atomicAdd(&fl->launches, 1ull);
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
  const FlagWords fw = load_flag_words(fl);
  const longlong2 sl = load_flag_pair(&fl->step);   // (step, step_limit)
  const bool active = fw.error == 0 && (sl.y < 0 || sl.x < sl.y);
  const int vfull = fw.v_full;

  bool need = false, bad = false;
  const int i = t.first + threadIdx.x;
  if (active && threadIdx.x < t.count) {
    // descriptor fields and every load first (no store may alias them), then math
    const int n = s.n;
    double* __restrict__ xp = s.x;
    double* __restrict__ vp = s.v;
    const double kick = vfull ? s.h : s.h + s.h;   // closing + opening half kicks
    const double dtq[3] = {s.dtq[0], s.dtq[1], s.dtq[2]};
    const float fsc[3] = {s.fscale[0], s.fscale[1], s.fscale[2]};
    const double Lr[3] = {s.L[0] * (1.0 / 4294967296.0), s.L[1] * (1.0 / 4294967296.0),
                          s.L[2] * (1.0 / 4294967296.0)};
    const float rb2 = s.rbuff_half2;
    int* __restrict__ imgp = s.img;
    int4* __restrict__ qp = s.q;
    double4_32a* __restrict__ p64p = s.p64;
    double f[3];
    if (PREC == GBMD_FP64) {
      const double4_32a F = s.f64[i];
      f[0] = F.x; f[1] = F.y; f[2] = F.z;
    } else {
      const float4 F = __ldg(s.f32 + i);
      f[0] = widen_f32(F.x, bad);
      f[1] = widen_f32(F.y, bad);
      f[2] = widen_f32(F.z, bad);
    }
    double v[3], xq[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      v[a] = vp[a * n + i];
      xq[a] = xp[a * n + i];
    }
    const int ty = __ldg(s.type + i);
    const int4 qb = __ldg(s.q_build + i);
    int q[3];
    double xr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      v[a] = fma(kick, f[a], v[a]);
      xq[a] = fma(dtq[a], v[a], xq[a]);
      long long qq = rint_ll(xq[a]);
      const long long k = (qq + 0x80000000LL) >> 32;       // floor((xq + 2^31) / 2^32)
      if (k != 0) {
        if (k > 1 || k < -1 || !isfinite(xq[a])) bad = true;
        xq[a] -= (double)k * 4294967296.0;
        qq -= k << 32;
        imgp[a * n + i] += (int)k;
      }
      q[a] = (int)qq;
      xr[a] = xq[a] * Lr[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      vp[a * n + i] = v[a];
      xp[a * n + i] = xq[a];
    }
    qp[i] = make_int4(q[0], q[1], q[2], ty);
    if (PREC == GBMD_FP64) p64p[i] = make_double4_32a(xr[0], xr[1], xr[2], __longlong_as_double(ty));
    const float dx = (float)min_image_fixed(q[0], qb.x) * fsc[0];
    const float dy = (float)min_image_fixed(q[1], qb.y) * fsc[1];
    const float dz = (float)min_image_fixed(q[2], qb.z) * fsc[2];
    need = dx * dx + dy * dy + dz * dz > rb2;
  }
  if (bad) atomicCAS(&fl->error, 0, (int)DEV_NONFINITE);   // rare: no block reduction
  const int any_need = __syncthreads_or(need);

  // ---- the last block to finish makes the per-step decisions ----
  // Only thread 0 publishes: its flag update, a fence, then the arrival count
  // (the position stores of this step need not be visible to the last block).
  __shared__ int last;
  if (threadIdx.x == 0) {
    if (any_need) atomicOr(&fl->rebuild_req, 1);
    __threadfence();
    last = (atomicAdd(&ctl->blocks_done, 1u) == gridDim.x - 1);
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
    if (act) {
      const long long st = sl.x + 1;
      const int rb = w.rebuild_req;
      const int srt = rb && sp > 0 && (st - lr.x >= sp);
      g->step = st;
      g->v_full = 0;
      g->rebuild_req = 0;
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

// ---------------------------------------------------------------------------
// K7: per-system thermo.  Sums the force kernel's per-tile partials (pe, W) and
// the kinetic term sum v^2 at full-step velocities, in a fixed order.
// thermo[0] = pe, thermo[1] = sum v^2, thermo[2..7] = W.
// ---------------------------------------------------------------------------
template <typename T>
__device__ double block_sum(double v, double* sh) {
  // fixed-order tree reduction over the block (deterministic)
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// U, sum v.v and W (6) of one system from the per-tile partial sums that the
// energy variant of the force kernel wrote just before (fixed order: each thread
// sums tiles t, t + 256, ... in order, then a fixed tree over the threads)
__global__ void __launch_bounds__(256) k_thermo(const SysDev* __restrict__ sysv,
                                                const Tile* __restrict__ tiles) {
  __shared__ double sh[256];
  const SysDev& s = sysv[tiles[blockIdx.x].sys];
  if (threadIdx.x == 0) atomicAdd(&s.flags->launches, 1ull);
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = threadIdx.x; k < s.tile_count_f; k += blockDim.x) {
    const double* p = s.partials + 8 * (size_t)(s.tile_first_f + k);
    for (int c = 0; c < 8; ++c) acc[c] += p[c];
  }
  double r = block_sum<double>(acc[7], sh);
  if (threadIdx.x == 0) s.thermo[1] = r;
  for (int c = 0; c < 7; ++c) {
    r = block_sum<double>(acc[c], sh);
    if (threadIdx.x == 0) s.thermo[c == 0 ? 0 : c + 1] = r;
  }
}

// ---------------------------------------------------------------------------
// import: tag-order row-major host layout -> internal planar arrays (identity order)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE_P) k_import(const SysDev* __restrict__ sysv,
                                                   const Tile* __restrict__ tiles,
                                                   const double* __restrict__ pos,
                                                   const double* __restrict__ vel,
                                                   const int* __restrict__ type,
                                                   const int* __restrict__ image) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  if (threadIdx.x >= t.count) return;
  const int i = t.first + threadIdx.x, n = s.n;
  int q[3];
  for (int a = 0; a < 3; ++a) {
    double x = pos[3 * (size_t)i + a];
    const double L = s.L[a];
    double k = floor((x + 0.5 * L) / L);   // centred box [-L/2, L/2)
    x -= k * L;
    if (x >= 0.5 * L) { x -= L; k += 1; }
    if (x < -0.5 * L) { x += L; k -= 1; }
    double xq = x * s.qscale[a];
    long long qq = __double2ll_rn(xq);
    if (qq >= 0x80000000LL) { xq -= 4294967296.0; qq -= 0x100000000LL; k += 1; }
    s.x[a * n + i] = xq;
    s.v[a * n + i] = vel[3 * (size_t)i + a];
    s.img[a * n + i] = (image ? image[3 * (size_t)i + a] : 0) + (int)k;
    q[a] = (int)qq;
  }
  int ty = type ? type[i] : 0;
  if ((unsigned)ty >= (unsigned)s.ntypes) {   // device-supplied types are checked here
    atomicCAS(&s.flags->error, 0, (int)DEV_BADTYPE);
    ty = 0;
  }
  s.type[i] = ty;
  s.tag[i] = i;
  s.rtag[i] = i;
  s.q[i] = make_int4(q[0], q[1], q[2], ty);
  s.q_build[i] = s.q[i];
  s.p64[i] = make_double4_32a(s.x[i] * (s.L[0] / 4294967296.0), s.x[n + i] * (s.L[1] / 4294967296.0),
                          s.x[2 * n + i] * (s.L[2] / 4294967296.0), __longlong_as_double(ty));
}

// ---------------------------------------------------------------------------
// export: internal arrays -> tag-order row-major (any output may be null)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE_P) k_export(const SysDev* __restrict__ sysv,
                                                   const Tile* __restrict__ tiles, double* pos,
                                                   double* vel, int* image, double* force,
                                                   double* pp_u, double* pp_w) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  if (threadIdx.x >= t.count) return;
  const int tg = t.first + threadIdx.x, n = s.n;
  const int i = s.rtag[tg];
  const int vfull = ((const volatile Flags*)s.flags)->v_full;
  double f[4];
  if (s.precision == GBMD_FP64) {
    double4_32a F = s.f64[i];
    f[0] = F.x; f[1] = F.y; f[2] = F.z; f[3] = F.w;
  } else {
    float4 F = s.f32[i];
    f[0] = F.x; f[1] = F.y; f[2] = F.z; f[3] = F.w;
  }
  for (int a = 0; a < 3; ++a) {
    if (pos) pos[3 * (size_t)tg + a] = s.x[a * n + i] * (s.L[a] / 4294967296.0);
    if (vel) {
      double v = s.v[a * n + i];
      if (!vfull) v = fma(s.h, f[a], v);
      vel[3 * (size_t)tg + a] = v;
    }
    if (image) image[3 * (size_t)tg + a] = s.img[a * n + i];
    if (force) force[3 * (size_t)tg + a] = f[a];
  }
  if (pp_u && s.pp_u) pp_u[tg] = s.pp_u[i];
  if (pp_w && s.pp_w)
    for (int c = 0; c < 6; ++c) pp_w[6 * (size_t)tg + c] = s.pp_w[6 * (size_t)i + c];
}

// ---------------------------------------------------------------------------
// neighbour rows -> tags, each row sorted ascending (diagnostic readout)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE_P) k_nlist_export(const SysDev* __restrict__ sysv,
                                                         const Tile* __restrict__ tiles,
                                                         int* counts, int* idx, int cap_out,
                                                         int* too_many) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  if (threadIdx.x >= t.count) return;
  const int tg = t.first + threadIdx.x;
  const int i = s.rtag[tg];
  const int nn = s.nn[i];
  counts[tg] = nn;
  if (nn > cap_out) {
    atomicExch(too_many, 1);
    return;
  }
  int* out = idx + (size_t)tg * cap_out;
  // staged lists hold window-local indices: map them back through the block's window
  const int2* bw = nullptr;
  const unsigned short* nl16 = reinterpret_cast<const unsigned short*>(s.nl);
  int m = 0;
  if (s.staged) {
    const int4 qb = s.q_build[i];
    const int cx = cell_of_fixed(qb.x, s.nc[0]), cy = cell_of_fixed(qb.y, s.nc[1]),
              cz = cell_of_fixed(qb.z, s.nc[2]);
    const int b = ((cz >> 1) * s.nb[1] + (cy >> 1)) * s.nb[0] + (cx >> 1);
    bw = s.blk_win + (size_t)b * WIN_CELLS;
    m = s.rmember[i];
  }
  for (int k = 0; k < nn; ++k) {   // insertion sort of the tags (rows are short)
    int j;
    if (s.staged) {
      const int local = nl16[nl16_index(m, k, s.nl_stride)];
      int c = 0;   // last window cell whose offset is <= local
      for (int step = 32; step > 0; step >>= 1)
        if (c + step < WIN_CELLS && bw[c + step].y <= local) c += step;
      j = s.members[bw[c].x + (local - bw[c].y)];
    } else {
      j = s.nl[nl_index(i, k, s.nl_stride)];
    }
    const int v = s.tag[j];
    int p = k;
    while (p > 0 && out[p - 1] > v) {
      out[p] = out[p - 1];
      --p;
    }
    out[p] = v;
  }
  for (int k = nn; k < cap_out; ++k) out[k] = -1;
}

// ---------------------------------------------------------------------------
// launch plumbing
// ---------------------------------------------------------------------------
template <typename T>
static void put(KernelCall& k, const T& v) {
  static_assert(sizeof(T) <= 16, "arg too large");
  memcpy(k.store[k.nargs], &v, sizeof(T));
  ++k.nargs;
}

static KernelCall mk(void* f, int grid, int block, size_t smem = 0) {
  KernelCall k;
  memset(&k, 0, sizeof(k));
  k.func = f;
  k.grid = dim3(grid > 0 ? grid : 1);
  k.block = dim3(block);
  k.smem = smem;
  return k;
}

cudaError_t launch(const KernelCall& k, cudaStream_t st) {
  void* a[10];
  args_of(k, a);
  return cudaLaunchKernel(k.func, k.grid, k.block, a, k.smem, st);
}

KernelCall integrate_call(int prec, const SysDev* d, const Tile* tiles, int ntiles, GroupCtl* ctl,
                          int nsys, cudaGraphConditionalHandle cond, int use_cond) {
  KernelCall k = mk(prec == GBMD_FP64 ? (void*)k_integrate<GBMD_FP64> : (void*)k_integrate<GBMD_MIXED>,
                    ntiles, TILE_P);
  put(k, d); put(k, tiles); put(k, ctl); put(k, nsys); put(k, cond); put(k, use_cond);
  return k;
}

KernelCall thermo_call(const SysDev* d, const Tile* tiles_s, int nsys, GroupCtl*) {
  KernelCall k = mk((void*)k_thermo, nsys, 256);
  put(k, d); put(k, tiles_s);
  return k;
}

KernelCall import_call(const SysDev* d, const Tile* tiles_p, int ntiles, const double* pos,
                       const double* vel, const int* type, const int* image) {
  KernelCall k = mk((void*)k_import, ntiles, TILE_P);
  put(k, d); put(k, tiles_p); put(k, pos); put(k, vel); put(k, type); put(k, image);
  return k;
}

KernelCall export_call(const SysDev* d, const Tile* tiles_p, int ntiles, double* pos, double* vel,
                       int* image, double* force, double* pp_u, double* pp_w) {
  KernelCall k = mk((void*)k_export, ntiles, TILE_P);
  put(k, d); put(k, tiles_p); put(k, pos); put(k, vel); put(k, image); put(k, force);
  put(k, pp_u); put(k, pp_w);
  return k;
}

KernelCall nlist_export_call(const SysDev* d, const Tile* tiles_p, int ntiles, int* counts,
                             int* idx, int cap_out, int* too_many) {
  KernelCall k = mk((void*)k_nlist_export, ntiles, TILE_P);
  put(k, d); put(k, tiles_p); put(k, counts); put(k, idx); put(k, cap_out); put(k, too_many);
  return k;
}

// shared with the other translation units
KernelCall make_call(void* f, int grid, int block, size_t smem) { return mk(f, grid, block, smem); }

}  // namespace gbmd
