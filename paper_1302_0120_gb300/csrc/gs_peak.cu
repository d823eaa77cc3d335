// gs_peak.cu -- measured FP32 fused multiply-add throughput of the device.
//
// A diagnostic: the paper has no counterpart. The iteration kernels do their
// arithmetic on the FP32 pipes, so the benchmark reports their throughput
// against this measured ceiling rather than a nominal one.
#include <cuda_runtime.h>

#include "gs.h"

namespace {

constexpr int kThreadsPeak = 256;
constexpr int kChains = 8;   // independent dependency chains per thread
constexpr int kUnroll = 16;  // FMAs per chain per round

__device__ float g_peak_sink;

// Every thread advances kChains independent chains x <- a x + b. With
// 0 < a < 1 and b > 0 every chain stays positive, so the store is never
// taken; the comparison still keeps the chains live.
__global__ void __launch_bounds__(kThreadsPeak) fma_peak_kernel(int rounds, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1e-6f * static_cast<float>(threadIdx.x) + static_cast<float>(j);
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == -1.0f) g_peak_sink = s;
}

}  // namespace

extern "C" int gs_fp32_peak(double* tflops_out, void* stream) {
  if (tflops_out == nullptr) return GS_EINVAL;
  *tflops_out = 0.0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GS_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel, kThreadsPeak, 0) != cudaSuccess)
    return GS_ECUDA;
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  const int rounds = 8192;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GS_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GS_ECUDA;
  }
  int rc = GS_OK;
  float best_ms = 0.f;
  for (int rep = 0; rep < 4 && rc == GS_OK; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, s);
    fma_peak_kernel<<<grid, kThreadsPeak, 0, s>>>(rounds, 0.999999f, 1e-6f);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = GS_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GS_OK) return rc;
  const double fmas = static_cast<double>(grid) * kThreadsPeak * kChains * kUnroll * rounds;
  *tflops_out = 2.0 * fmas / (best_ms * 1e-3) / 1e12;
  return GS_OK;
}
