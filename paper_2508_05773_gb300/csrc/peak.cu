// peak.cu -- issue-rate microbenchmarks of the SM pipes the solve uses
// (FP32 fused multiply-add, integer multiply-add, the XU's reciprocal
// square root), for the roofline denominators.  Each thread runs eight
// independent dependency chains, so that with full occupancy the pipe,
// not latency, bounds the rate.  Nothing here changes a GPU setting.
#include <cstdint>

#include "brmppi.h"
#include "internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

// where the kernels would write their (never produced) results: keeps the
// chains live without a caller buffer
__device__ uint32_t g_sink[4096];

__global__ void __launch_bounds__(512) pipe_fma_kernel(long long iters, float b, float c, float* sink) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1.0f + 1e-7f * static_cast<float>(threadIdx.x + 37 * j);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
  }
  float r = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) r += a[j];
  if (r == 1234.5f) sink[blockIdx.x] = r;  // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(512) pipe_imad_kernel(long long iters, uint32_t m, uint32_t c, uint32_t* sink) {
  uint32_t a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = threadIdx.x * 2654435761u + static_cast<uint32_t>(j);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = a[j] * m + c;
  }
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) r ^= a[j];
  if (r == 0x9E3779B9u && c == 0u) sink[blockIdx.x] = r;
}

__global__ void __launch_bounds__(512) pipe_xu_kernel(long long iters, float c, float* sink) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1.0f + 1e-3f * static_cast<float>(j);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = rsqrtf(a[j]) + c;  // MUFU.RSQ, then the add
  }
  float r = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) r += a[j];
  if (r == 1234.5f) sink[blockIdx.x] = r;
}

}  // namespace

extern "C" brmppi_status brmppi_measure_pipe(int32_t pipe, int64_t iters, double* lane_ops_per_s, double* seconds,
                                             void* stream) {
  using namespace brmppi_host;
  if (!lane_ops_per_s || iters < 1 || pipe < 0 || pipe > 2) return fail(nullptr, BRMPPI_EINVAL, "bad argument");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "device query");
  const int threads = 512, blocks = 4 * sms;  // 2048 threads a SM: every warp slot filled
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* sink = nullptr;
  if ((e = cudaGetSymbolAddress(&sink, g_sink)) != cudaSuccess) return cuda_fail(nullptr, e, "sink");
  if (blocks > 4096) return fail(nullptr, BRMPPI_EINVAL, "too many SMs for the sink");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(nullptr, e, "cudaEventCreate");
  }
  auto launch = [&](long long n) {
    if (pipe == 0)
      pipe_fma_kernel<<<blocks, threads, 0, s>>>(n, 0.9999999f, 1e-7f, static_cast<float*>(sink));
    else if (pipe == 1)
      pipe_imad_kernel<<<blocks, threads, 0, s>>>(n, 1664525u, 1013904223u, static_cast<uint32_t*>(sink));
    else
      pipe_xu_kernel<<<blocks, threads, 0, s>>>(n, 0.5f, static_cast<float*>(sink));
  };
  launch(iters / 16 + 1);  // warm-up
  cudaEventRecord(e0, s);
  launch(iters);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "pipe microbenchmark");
  // lane operations: the pipe's instruction per chain step (the XU kernel
  // also issues one FP32 add per step, not counted)
  const double ops = static_cast<double>(blocks) * threads * static_cast<double>(iters) * kUnroll * kChains;
  *lane_ops_per_s = ops / (1e-3 * ms);
  if (seconds) *seconds = 1e-3 * ms;
  return BRMPPI_OK;
}
