// gs_loss_inst.cu -- instantiations and launch of the loss/adjoint kernel
// (square grids, log2 n in [5, 12]).
#include "gs_loss.cuh"

namespace gsk {

template <int MODE>
static const void* loss_kernel_mode(int logn) {
  switch (logn) {
    case 5: return reinterpret_cast<const void*>(gs_loss_kernel<5, MODE>);
    case 6: return reinterpret_cast<const void*>(gs_loss_kernel<6, MODE>);
    case 7: return reinterpret_cast<const void*>(gs_loss_kernel<7, MODE>);
    case 8: return reinterpret_cast<const void*>(gs_loss_kernel<8, MODE>);
    case 9: return reinterpret_cast<const void*>(gs_loss_kernel<9, MODE>);
    case 10: return reinterpret_cast<const void*>(gs_loss_kernel<10, MODE>);
    case 11: return reinterpret_cast<const void*>(gs_loss_kernel<11, MODE>);
    case 12: return reinterpret_cast<const void*>(gs_loss_kernel<12, MODE>);
    default: return nullptr;
  }
}

static const void* loss_kernel_for(int logn, int mode) {
  return mode == kLossPrepare ? loss_kernel_mode<kLossPrepare>(logn)
         : mode == kLossStep  ? loss_kernel_mode<kLossStep>(logn)
                              : loss_kernel_mode<kLossFused>(logn);
}

cudaError_t launch_loss(const LossParams& p, int grid, cudaStream_t s) {
  const void* k = loss_kernel_for(p.logn, p.mode);
  if (k == nullptr) return cudaErrorInvalidValue;
  const size_t smem = iteration_smem_bytes(p.n, p.n);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (grid > per_sm * sms) grid = per_sm * sms;
  if (grid < 1) grid = 1;
  void* args[] = {const_cast<LossParams*>(&p)};
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kThreads), args, smem, s);
}

}  // namespace gsk
