// gs_rg_inst.cu -- the register-resident iteration kernels for grids whose
// sides are 600 or 800 (gs_rg.cuh), one per pair of sides.
#include "gs_iterate.cuh"

namespace gsk {

template <int NX, int NY>
__global__ void __launch_bounds__(kThreads, 1) gs_iterate_rg(const Params p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shared sh;
  if (*reinterpret_cast<volatile int*>(p.abort_flag) != 0) return;  // an earlier chunk failed
  const StageTw<5> none{};
  iterate_class<NX, NY, false>(p, sh, smem, none, NoTc{});
}

const void* iterate_kernel_rg(int nx, int ny) {
  if (nx == 800 && ny == 600) return reinterpret_cast<const void*>(gs_iterate_rg<800, 600>);
  if (nx == 600 && ny == 800) return reinterpret_cast<const void*>(gs_iterate_rg<600, 800>);
  if (nx == 800 && ny == 800) return reinterpret_cast<const void*>(gs_iterate_rg<800, 800>);
  if (nx == 600 && ny == 600) return reinterpret_cast<const void*>(gs_iterate_rg<600, 600>);
  return nullptr;
}

size_t rg_smem_bytes(int nx, int ny) {
  if (nx == 800 && ny == 600) return RgSmem<800, 600>::kBytes;
  if (nx == 600 && ny == 800) return RgSmem<600, 800>::kBytes;
  if (nx == 800 && ny == 800) return RgSmem<800, 800>::kBytes;
  if (nx == 600 && ny == 600) return RgSmem<600, 600>::kBytes;
  return 0;
}

}  // namespace gsk
