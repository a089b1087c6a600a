// Rate probes for the roofline denominators that no driver measurement provides: the FP64 FMA
// rate of the device (the bound of the FP64 iteration kernels' arithmetic) and the read bandwidth
// of a buffer resident in L2 (the bound of the iteration kernels on LPs whose working set fits in
// L2).  Both time their kernel with CUDA events on the caller's stream after a warm-up launch and
// report the best of several launches.  They change no device setting.
#include <cuda_runtime.h>

#include <string>

#include "../../include/rhpdhg.h"
#include "internal.h"

namespace rh {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kFmaChains = 8;       // independent FMA chains per thread

// Each thread runs kFmaChains independent chains x <- x * a + b for `iters` rounds; the values
// stay in [0.5, 2] (a < 1, b chosen so the fixed point is 1), so no denormal or overflow slows
// the pipe.  The result is stored only under a condition that never holds, which keeps the
// chains alive without a store per thread.
__global__ void __launch_bounds__(kProbeThreads)
k_fp64_fma(int iters, double a, double b, double *sink) {
  double x[kFmaChains];
#pragma unroll
  for (int u = 0; u < kFmaChains; ++u) x[u] = 1.0 + 1e-3 * (threadIdx.x + u);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kFmaChains; ++u) x[u] = fma(x[u], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < kFmaChains; ++u) s += x[u];
  if (s == -1.0) sink[blockIdx.x] = s;
}

// Grid-stride read of n 16-byte words; the XOR of what each thread read is stored under a
// condition that never holds.
__global__ void __launch_bounds__(kProbeThreads)
k_read(const uint4 *__restrict__ p, long long n, unsigned *sink) {
  unsigned acc = 0u;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    const uint4 a = __ldcg(p + i), b = __ldcg(p + i + stride), c = __ldcg(p + i + 2 * stride),
                d = __ldcg(p + i + 3 * stride);
    acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^
           d.z ^ d.w;
  }
  for (; i < n; i += stride) {
    const uint4 a = __ldcg(p + i);
    acc ^= a.x ^ a.y ^ a.z ^ a.w;
  }
  if (acc == 0xFFFFFFFFu) sink[blockIdx.x] = acc;
}

// Best of `reps` timed launches of fn (after one untimed launch), in milliseconds.
template <typename Fn>
cudaError_t time_best(cudaStream_t st, int reps, Fn fn, float *best_ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  e = fn();
  float best = 1e30f;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_ms = best;
  return e;
}

int probe_fail(const char *who, cudaError_t e) {
  set_global_error(std::string(who) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? RHPDHG_ERR_OOM : RHPDHG_ERR_CUDA;
}

}  // namespace

}  // namespace rh

extern "C" int rhpdhg_probe_fp64_fma_rate(void *cuda_stream, double *tflops) {
  using namespace rh;
  if (!tflops) {
    set_global_error("rhpdhg_probe_fp64_fma_rate: tflops is NULL");
    return RHPDHG_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, kProbeThreads, 0);
  if (e != cudaSuccess) return probe_fail("rhpdhg_probe_fp64_fma_rate", e);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  const int iters = 4096;
  double *sink = nullptr;
  e = cudaMalloc(&sink, (size_t)grid * sizeof(double));
  if (e != cudaSuccess) return probe_fail("rhpdhg_probe_fp64_fma_rate", e);
  const double a = 0.999, b = 0.001;     // fixed point 1
  float ms = 0.f;
  e = time_best(st, 5, [&]() {
    return launch_kernel(k_fp64_fma, grid, kProbeThreads, 0, st, iters, a, b, sink);
  }, &ms);
  cudaFree(sink);
  if (e != cudaSuccess) return probe_fail("rhpdhg_probe_fp64_fma_rate", e);
  count_launches(6);
  const double flops = 2.0 * kFmaChains * (double)iters * grid * kProbeThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return RHPDHG_OK;
}

extern "C" int rhpdhg_probe_l2_read_bandwidth(int64_t bytes, void *cuda_stream, double *gbs) {
  using namespace rh;
  if (!gbs || bytes < (1 << 20) || bytes > (1LL << 32)) {
    set_global_error("rhpdhg_probe_l2_read_bandwidth: gbs is NULL or bytes outside [1 MiB, 4 GiB]");
    return RHPDHG_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_read, kProbeThreads, 0);
  if (e != cudaSuccess) return probe_fail("rhpdhg_probe_l2_read_bandwidth", e);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  const long long words = bytes / 16;
  uint4 *buf = nullptr;
  unsigned *sink = nullptr;
  e = cudaMalloc(&buf, (size_t)words * 16);
  if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)grid * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 1, (size_t)words * 16, st);
  float ms = 0.f;
  if (e == cudaSuccess)
    e = time_best(st, 10, [&]() {
      return launch_kernel(k_read, grid, kProbeThreads, 0, st, (const uint4 *)buf, words, sink);
    }, &ms);
  cudaStreamSynchronize(st);
  cudaFree(buf);
  cudaFree(sink);
  if (e != cudaSuccess) return probe_fail("rhpdhg_probe_l2_read_bandwidth", e);
  count_launches(11);
  *gbs = (double)words * 16.0 / (ms * 1e-3) / 1e9;
  return RHPDHG_OK;
}
