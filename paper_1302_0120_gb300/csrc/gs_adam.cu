// gs_adam.cu -- one Adam update of a phase mask (the optimiser of the
// differentiable form), as a grid-stride elementwise kernel.
#include <cuda_runtime.h>

#include <cmath>

#include "gs.h"

namespace {

constexpr int kAdamThreads = 256;

// p -= (lr / b1) m / (sqrt(v) / sqrt(b2) + eps) with m, v the running first
// and second moments of the gradient and b1, b2 the bias corrections
// 1 - beta^t of step t = state[0] + 1. The last block to finish advances
// state[0] (every block has read it by then) and rearms the counter state[1].
__global__ void __launch_bounds__(kAdamThreads) adam_kernel(float* __restrict__ phase, const float* __restrict__ grad,
                                                            float* __restrict__ m, float* __restrict__ v, long long n,
                                                            int* state, float lr, float beta1, float beta2, float eps) {
  const int t = state[0] + 1;
  const float b1 = 1.f - powf(beta1, static_cast<float>(t));
  const float b2 = 1.f - powf(beta2, static_cast<float>(t));
  const float step = lr / b1;
  const float rb2 = 1.f / sqrtf(b2);
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float g = grad[i];
    const float mi = fmaf(beta1, m[i], (1.f - beta1) * g);
    const float vi = fmaf(beta2, v[i], (1.f - beta2) * g * g);
    m[i] = mi;
    v[i] = vi;
    phase[i] -= step * mi / (sqrtf(vi) * rb2 + eps);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(state + 1, 1) == static_cast<int>(gridDim.x) - 1) {
      state[0] = t;
      state[1] = 0;
    }
  }
}

}  // namespace

extern "C" int gs_adam_step(float* phase, const float* grad, float* m, float* v, long long n, int* state, float lr,
                            float beta1, float beta2, float eps, void* stream) {
  if (phase == nullptr || grad == nullptr || m == nullptr || v == nullptr || state == nullptr || n < 1 ||
      !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return GS_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  long long blocks = (n + kAdamThreads - 1) / kAdamThreads;
  if (blocks > 8LL * sms) blocks = 8LL * sms;
  adam_kernel<<<static_cast<int>(blocks), kAdamThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      phase, grad, m, v, n, state, lr, beta1, beta2, eps);
  if (cudaGetLastError() != cudaSuccess) return GS_ECUDA;
  return GS_OK;
}
