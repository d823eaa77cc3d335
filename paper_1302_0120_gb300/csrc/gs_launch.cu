// gs_launch.cu -- host helpers that select, size and launch the iteration kernel.
#include <cfloat>

#include "gs_internal.h"

namespace gsk {

// sum p^2 in FP64 by one block in a fixed order; NaN if any p is negative or
// not finite.
__global__ void __launch_bounds__(1024) energy_kernel(const float* __restrict__ p, long long n, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  bool bad = false;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    const float x = p[e];
    bad |= !(x >= 0.f && x <= FLT_MAX);
    acc += static_cast<double>(x) * static_cast<double>(x);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  const int any_bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
    out[0] = any_bad ? __longlong_as_double(0x7ff8000000000000ll) : s;
  }
}

cudaError_t launch_energy(const float* p, long long n, double* energy, cudaStream_t s) {
  energy_kernel<<<1, 1024, 0, s>>>(p, n, energy);
  return cudaGetLastError();
}

// Each is defined in the gs_inst.cu object compiled with GS_LX = LX.
extern template const void* iterate_kernel_lx<5>(int);
extern template const void* iterate_kernel_lx<6>(int);
extern template const void* iterate_kernel_lx<7>(int);
extern template const void* iterate_kernel_lx<8>(int);
extern template const void* iterate_kernel_lx<9>(int);
extern template const void* iterate_kernel_lx<10>(int);
extern template const void* iterate_kernel_lx<11>(int);
extern template const void* iterate_kernel_lx<12>(int);

extern template const void* iterate_kernel_rg_nx<600>(int);
extern template const void* iterate_kernel_rg_nx<768>(int);
extern template const void* iterate_kernel_rg_nx<800>(int);
extern template const void* iterate_kernel_rg_nx<1024>(int);
extern template size_t rg_smem_bytes_nx<600>(int);
extern template size_t rg_smem_bytes_nx<768>(int);
extern template size_t rg_smem_bytes_nx<800>(int);
extern template size_t rg_smem_bytes_nx<1024>(int);

const void* iterate_kernel_rg(int nx, int ny) {
  switch (nx) {
    case 600: return iterate_kernel_rg_nx<600>(ny);
    case 768: return iterate_kernel_rg_nx<768>(ny);
    case 800: return iterate_kernel_rg_nx<800>(ny);
    case 1024: return iterate_kernel_rg_nx<1024>(ny);
    default: return nullptr;
  }
}

size_t rg_smem_bytes(int nx, int ny) {
  switch (nx) {
    case 600: return rg_smem_bytes_nx<600>(ny);
    case 768: return rg_smem_bytes_nx<768>(ny);
    case 800: return rg_smem_bytes_nx<800>(ny);
    case 1024: return rg_smem_bytes_nx<1024>(ny);
    default: return 0;
  }
}

static int log2_exact(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

static const void* kernel_for(int nx, int ny, int tc_mode) {
  if (uses_general(nx, ny)) {
    if (tc_mode != kTcNone) return nullptr;
    return uses_rg(nx, ny) ? iterate_kernel_rg(nx, ny) : iterate_kernel_general();
  }
  const int ly = log2_exact(ny);
  if (tc_mode == kTcGen05F16 || tc_mode == kTcGen05Bf16)
    return nx == ny ? iterate_kernel_tc5(ly, tc_mode == kTcGen05Bf16) : nullptr;
  if (tc_mode == kTcMmaSync) return nx == ny ? iterate_kernel_tc(ly) : nullptr;
  switch (log2_exact(nx)) {
    case 5: return iterate_kernel_lx<5>(ly);
    case 6: return iterate_kernel_lx<6>(ly);
    case 7: return iterate_kernel_lx<7>(ly);
    case 8: return iterate_kernel_lx<8>(ly);
    case 9: return iterate_kernel_lx<9>(ly);
    case 10: return iterate_kernel_lx<10>(ly);
    case 11: return iterate_kernel_lx<11>(ly);
    case 12: return iterate_kernel_lx<12>(ly);
    default: return nullptr;
  }
}

size_t iteration_smem_bytes(int nx, int ny, int tc_mode) {
  if (uses_rg(nx, ny)) return rg_smem_bytes(nx, ny);
  if (uses_general(nx, ny)) return gen_smem_bytes(nx, ny);
  // group exchange buffers, one column block of the amplitude, one of the
  // field; then the tensor-core tables (and, for tcgen05, operands)
  const size_t extra = tc_mode == kTcMmaSync ? kTcExtraSmemBytes
                       : (tc_mode == kTcGen05F16 || tc_mode == kTcGen05Bf16) ? kTc5ExtraSmemBytes
                                                                               : 0;
  return kGroupSmemBytes + 8192 * 4 + 8192 * 8 + extra;
}

cudaError_t iteration_occupancy(int nx, int ny, int* blocks_per_sm, int tc_mode) {
  const void* k = kernel_for(nx, ny, tc_mode);
  if (k == nullptr) return cudaErrorInvalidValue;
  const size_t smem = iteration_smem_bytes(nx, ny, tc_mode);
  // The general kernel serves every size: allow its largest request, so that
  // contexts of different sizes do not undo each other's setting.
  const size_t allow = (uses_general(nx, ny) && !uses_rg(nx, ny)) ? gen_smem_bytes(kMaxGeneralSide, kMaxGeneralSide) : smem;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(allow));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kThreads, smem);
}

size_t mixed_smem_bytes(int tc_mode) {
  // mma.sync: one twiddle table per class, then the shared cos/sin table;
  // tcgen05: the matrices and twiddle tables of the three lengths
  const size_t extra = tc_mode == kTcMmaSync ? 3 * 32 * 32 * 8 + 32 * 8
                       : (tc_mode == kTcGen05F16 || tc_mode == kTcGen05Bf16) ? kMixedTc5ExtraSmemBytes
                                                                               : 0;
  return kGroupSmemBytes + 8192 * 4 + 8192 * 8 + extra;
}

cudaError_t mixed_occupancy(int tc_mode, int* blocks_per_sm) {
  const void* k = iterate_kernel_mixed(tc_mode);
  const size_t smem = mixed_smem_bytes(tc_mode);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kThreads, smem);
}

cudaError_t launch_mixed(const MixedParams& mp, int grid, int tc_mode, cudaStream_t s) {
  void* args[] = {const_cast<MixedParams*>(&mp)};
  return cudaLaunchCooperativeKernel(iterate_kernel_mixed(tc_mode), dim3(grid), dim3(kThreads), args,
                                     mixed_smem_bytes(tc_mode), s);
}

cudaError_t launch_iterations(const Params& p, int grid, cudaStream_t s) {
  const void* k = kernel_for(p.nx, p.ny, p.tensor_core);
  if (k == nullptr) return cudaErrorInvalidValue;
  const size_t smem = iteration_smem_bytes(p.nx, p.ny, p.tensor_core);
  void* args[] = {const_cast<Params*>(&p)};
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kThreads), args, smem, s);
}

}  // namespace gsk
