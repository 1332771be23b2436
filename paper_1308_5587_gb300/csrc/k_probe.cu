// k_probe.cu -- throughput probe of the arithmetic the force kernels lean on: the
// denominator of the FP64 force path's roofline (that path is bound by the FP64
// pipe, not by memory) and the FP32 rate it is compared with.
//
// Every thread runs CH independent chains of one operation for `iters` rounds, so
// the pipe, not latency, sets the rate:
//   PROBE_DFMA: x <- fma(x, a, b) in FP64          (one FP64 multiply-add)
//   PROBE_FFMA: x <- fmaf(x, a, b) in FP32         (one FP32 multiply-add)
//   PROBE_DRCP: x <- rcp_f64(x) in FP64            (the reciprocal the FP64 pair
//                                                   force takes once per pair)
// The grid is the SM count times 8 blocks of 256 threads.  Each thread stores the
// sum of its chains, so the compiler cannot drop them.
#include "launch.cuh"
#include "fp64_math.cuh"

namespace gbmd {

constexpr int PROBE_CH = 8;
constexpr int PROBE_BLOCK = 256;

template <int KIND>
__global__ void __launch_bounds__(PROBE_BLOCK) k_probe(double* __restrict__ sink, int iters,
                                                       double a, double b) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if constexpr (KIND == GBMD_PROBE_FFMA) {
    float x[PROBE_CH];
    const float af = (float)a, bf = (float)b;
#pragma unroll
    for (int c = 0; c < PROBE_CH; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
      for (int c = 0; c < PROBE_CH; ++c) x[c] = fmaf(x[c], af, bf);
    }
#pragma unroll
    for (int c = 0; c < PROBE_CH; ++c) acc += (double)x[c];
  } else {
    double x[PROBE_CH];
#pragma unroll
    for (int c = 0; c < PROBE_CH; ++c) x[c] = 1.0 + 1e-3 * (double)(threadIdx.x + c);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
      for (int c = 0; c < PROBE_CH; ++c) {
        if constexpr (KIND == GBMD_PROBE_DFMA) x[c] = fma(x[c], a, b);
        else x[c] = rcp_f64(x[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < PROBE_CH; ++c) acc += x[c];
  }
  sink[tid] = acc;
}

// one timed run of `iters` rounds on every SM; returns the operations executed and
// the event time of the launch on `st`
cudaError_t probe_run(int kind, cudaStream_t st, int iters, double* ops, float* ms) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = sms * 8;
  void* f = kind == GBMD_PROBE_FFMA ? (void*)k_probe<GBMD_PROBE_FFMA>
            : kind == GBMD_PROBE_DRCP ? (void*)k_probe<GBMD_PROBE_DRCP>
                                      : (void*)k_probe<GBMD_PROBE_DFMA>;
  double* sink = nullptr;
  e = cudaMalloc(&sink, sizeof(double) * (size_t)grid * PROBE_BLOCK);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double a = 0.999999, b = 1e-7;
  int warm = 16;
  void* args_w[] = {&sink, &warm, &a, &b};
  void* args[] = {&sink, &iters, &a, &b};
  if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess &&
      (e = cudaLaunchKernel(f, dim3(grid), dim3(PROBE_BLOCK), args_w, 0, st)) == cudaSuccess &&
      (e = cudaEventRecord(e0, st)) == cudaSuccess &&
      (e = cudaLaunchKernel(f, dim3(grid), dim3(PROBE_BLOCK), args, 0, st)) == cudaSuccess &&
      (e = cudaEventRecord(e1, st)) == cudaSuccess &&
      (e = cudaEventSynchronize(e1)) == cudaSuccess)
    e = cudaEventElapsedTime(ms, e0, e1);
  *ops = (double)grid * PROBE_BLOCK * (double)iters * PROBE_CH;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaError_t ef = cudaFree(sink);
  return e != cudaSuccess ? e : ef;
}

}  // namespace gbmd
