// k_step.cu -- thermo reduction and the import/export kernels of the C ABI.
//
// Velocity Verlet (NVE; Listing 1's mode_standard(dt) + run(n), NVE per Section 3.1):
//   v <- v + dt/(2m) F(t);  x <- x + dt v;  wrap;  F(t+dt);  v <- v + dt/(2m) F(t+dt).
// The step kernel (k_force in step mode, step_core.cuh) computes F(x^n) and then
// applies the closing half kick of step n-1 and the opening half kick of step n back
// to back, so the stored velocity lags half a kick behind the full-step velocity
// between steps (Flags::v_full says when it does not, i.e. right after create /
// set_state); readouts add h F(x^n) with the force at the current positions.
// Positions are stored in FP64 in units of L/2^32 per axis (xq = x * 2^32 / L).
#include <cstring>

#include "launch.cuh"

namespace gbmd {

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
// set_state, before anything is replaced: whether the new positions and velocities
// (tag order, in the staging buffers) are all finite, and the current types in tag
// order for the import
__global__ void __launch_bounds__(TILE_P) k_prep_state(const SysDev* __restrict__ sysv,
                                                       const Tile* __restrict__ tiles,
                                                       const double* __restrict__ pos,
                                                       const double* __restrict__ vel,
                                                       int* __restrict__ type_by_tag, int* bad) {
  const Tile t = tiles[blockIdx.x];
  const SysDev& s = sysv[t.sys];
  if (threadIdx.x >= t.count) return;
  const int g = t.first + threadIdx.x;   // a tag
  bool ok = true;
  for (int a = 0; a < 3; ++a)
    ok = ok && isfinite(pos[3 * (size_t)g + a]) && isfinite(vel[3 * (size_t)g + a]);
  if (!ok) atomicExch(bad, 1);
  type_by_tag[g] = s.type[s.rtag[g]];
}

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
  // both shadow buffers: the step counter is set after the import
  const int4 qn = make_int4(q[0], q[1], q[2], ty);
  s.q[i] = qn;
  s.q1[i] = qn;
  s.q_build[i] = qn;
  if (s.precision == GBMD_FP64) {   // the FP64 gather copies exist in FP64 mode only
    const double4_32a pn = make_double4_32a(s.x[i] * (s.L[0] / 4294967296.0), s.x[n + i] * (s.L[1] / 4294967296.0),
                                            s.x[2 * n + i] * (s.L[2] / 4294967296.0), __longlong_as_double(ty));
    s.p64[i] = pn;
    s.p64b[i] = pn;
  }
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
      if (!vfull) {
        v = fma(s.h, f[a], v);
        if (s.nvt) v *= s.nh[2];   // NVT: the closing thermostat scaling
      }
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
// domain decomposition: ghost positions in, selected positions out
// ---------------------------------------------------------------------------
// ghost k (tag n - n_ghost + k) takes pos[k] (row-major, real units, any image):
// x, the current step's shadow and, in FP64, its gather copy; the image counts of a
// ghost are not kept
__global__ void __launch_bounds__(TILE_P) k_ghost_set(const SysDev* __restrict__ d,
                                                      const double* __restrict__ pos) {
  const SysDev& s = *d;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= s.n_ghost) return;
  const int n = s.n;
  const int i = s.rtag[n - s.n_ghost + k];
  const long long step = step_of(s.flags);
  int q[3];
  double xr[3];
  for (int a = 0; a < 3; ++a) {
    const double L = s.L[a];
    double x = pos[3 * (size_t)k + a];
    x -= floor((x + 0.5 * L) / L) * L;   // centred box [-L/2, L/2)
    if (x >= 0.5 * L) x -= L;
    if (x < -0.5 * L) x += L;
    double xq = x * s.qscale[a];
    long long qq = __double2ll_rn(xq);
    if (qq >= 0x80000000LL) { xq -= 4294967296.0; qq -= 0x100000000LL; }
    s.x[a * n + i] = xq;
    q[a] = (int)qq;
    xr[a] = xq * (L / 4294967296.0);
  }
  const int ty = s.type[i];
  q_at(s, step)[i] = make_int4(q[0], q[1], q[2], ty);
  if (s.precision == GBMD_FP64)
    p64_at(s, step)[i] = make_double4_32a(xr[0], xr[1], xr[2], __longlong_as_double(ty));
}

// out[k] = the wrapped position of the particle with tag tags[k] (NaN for a tag out
// of range)
__global__ void __launch_bounds__(TILE_P) k_gather_pos(const SysDev* __restrict__ d,
                                                       const int* __restrict__ tags, int m,
                                                       double* __restrict__ out) {
  const SysDev& s = *d;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int tg = tags[k], n = s.n;
  const bool ok = tg >= 0 && tg < n;
  const int i = ok ? s.rtag[tg] : 0;
  for (int a = 0; a < 3; ++a)
    out[3 * (size_t)k + a] = ok ? s.x[a * n + i] * (s.L[a] / 4294967296.0) : __longlong_as_double(0x7ff8000000000000LL);
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

KernelCall prep_state_call(const SysDev* d, const Tile* tiles_p, int ntiles, const double* pos,
                           const double* vel, int* type_by_tag, int* bad) {
  KernelCall k = mk((void*)k_prep_state, ntiles, TILE_P);
  put(k, d); put(k, tiles_p); put(k, pos); put(k, vel); put(k, type_by_tag); put(k, bad);
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

KernelCall ghost_set_call(const SysDev* d, int n_ghost, const double* pos) {
  KernelCall k = mk((void*)k_ghost_set, (n_ghost + TILE_P - 1) / TILE_P, TILE_P);
  put(k, d); put(k, pos);
  return k;
}

KernelCall gather_pos_call(const SysDev* d, const int* tags, int m, double* out) {
  KernelCall k = mk((void*)k_gather_pos, (m + TILE_P - 1) / TILE_P, TILE_P);
  put(k, d); put(k, tags); put(k, m); put(k, out);
  return k;
}

// shared with the other translation units
KernelCall make_call(void* f, int grid, int block, size_t smem) { return mk(f, grid, block, smem); }

}  // namespace gbmd
