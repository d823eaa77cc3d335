// gs_rg_inst.cu -- the register-resident iteration kernels (gs_rg.cuh), one
// per pair of sides.
//
// Compiled once per row length nx in {600, 768, 800, 1024} with
// -DGS_RG_NX=<nx>; each object provides iterate_kernel_rg_nx<GS_RG_NX>(ny)
// and rg_smem_bytes_nx<GS_RG_NX>(ny) for every column length ny of the same
// set (1024 x 1024 excepted: it runs on the power-of-two kernel).
#include "gs_iterate.cuh"

#ifndef GS_RG_NX
#error "GS_RG_NX must be defined (the row length)"
#endif

namespace gsk {

template <int NX, int NY>
__global__ void __launch_bounds__(kThreads, 1) gs_iterate_rg(const Params p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shared sh;
  if (*reinterpret_cast<volatile int*>(p.abort_flag) != 0) return;  // an earlier chunk failed
  const StageTw<5> none{};
  iterate_class<NX, NY, false>(p, sh, smem, none, NoTc{});
}

template <>
const void* iterate_kernel_rg_nx<GS_RG_NX>(int ny) {
  switch (ny) {
    case 600: return reinterpret_cast<const void*>(gs_iterate_rg<GS_RG_NX, 600>);
    case 768: return reinterpret_cast<const void*>(gs_iterate_rg<GS_RG_NX, 768>);
    case 800: return reinterpret_cast<const void*>(gs_iterate_rg<GS_RG_NX, 800>);
#if GS_RG_NX != 1024
    case 1024: return reinterpret_cast<const void*>(gs_iterate_rg<GS_RG_NX, 1024>);
#endif
    default: return nullptr;
  }
}

template <>
size_t rg_smem_bytes_nx<GS_RG_NX>(int ny) {
  switch (ny) {
    case 600: return RgSmem<GS_RG_NX, 600>::kBytes;
    case 768: return RgSmem<GS_RG_NX, 768>::kBytes;
    case 800: return RgSmem<GS_RG_NX, 800>::kBytes;
#if GS_RG_NX != 1024
    case 1024: return RgSmem<GS_RG_NX, 1024>::kBytes;
#endif
    default: return 0;
  }
}

}  // namespace gsk
