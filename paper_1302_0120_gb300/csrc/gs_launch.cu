// gs_launch.cu -- host helpers that select, size and launch the iteration kernel.
#include "gs_internal.h"

namespace gsk {

// Each is defined in the gs_inst.cu object compiled with GS_LX = LX.
extern template const void* iterate_kernel_lx<5>(int);
extern template const void* iterate_kernel_lx<6>(int);
extern template const void* iterate_kernel_lx<7>(int);
extern template const void* iterate_kernel_lx<8>(int);
extern template const void* iterate_kernel_lx<9>(int);
extern template const void* iterate_kernel_lx<10>(int);
extern template const void* iterate_kernel_lx<11>(int);
extern template const void* iterate_kernel_lx<12>(int);

static int log2_exact(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

static const void* kernel_for(int nx, int ny) {
  const int ly = log2_exact(ny);
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

size_t iteration_smem_bytes(int nx, int ny) {
  (void)nx;
  (void)ny;
  // group exchange buffers, one column block of the amplitude, one of the field
  return kGroupSmemBytes + 8192 * 4 + 8192 * 8;
}

cudaError_t iteration_occupancy(int nx, int ny, int* blocks_per_sm) {
  const void* k = kernel_for(nx, ny);
  if (k == nullptr) return cudaErrorInvalidValue;
  const size_t smem = iteration_smem_bytes(nx, ny);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kThreads, smem);
}

cudaError_t launch_iterations(const Params& p, int grid, cudaStream_t s) {
  const void* k = kernel_for(p.nx, p.ny);
  if (k == nullptr) return cudaErrorInvalidValue;
  const size_t smem = iteration_smem_bytes(p.nx, p.ny);
  void* args[] = {const_cast<Params*>(&p)};
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kThreads), args, smem, s);
}

}  // namespace gsk
