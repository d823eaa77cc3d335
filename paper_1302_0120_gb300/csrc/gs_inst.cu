// gs_inst.cu -- instantiations of the iteration kernel for one log2(nx).
//
// Compiled once per log2(nx) in [5, 12] with -DGS_LX=<value>; each object
// provides iterate_kernel_lx<GS_LX>(log2 ny) for every log2(ny) in [5, 12].
#include "gs_iterate.cuh"

#ifndef GS_LX
#error "GS_LX must be defined (log2 of nx)"
#endif

namespace gsk {

template <>
const void* iterate_kernel_lx<GS_LX>(int ly) {
  switch (ly) {
    case 5: return reinterpret_cast<const void*>(gs_iterate<GS_LX, 5>);
    case 6: return reinterpret_cast<const void*>(gs_iterate<GS_LX, 6>);
    case 7: return reinterpret_cast<const void*>(gs_iterate<GS_LX, 7>);
    case 8: return reinterpret_cast<const void*>(gs_iterate<GS_LX, 8>);
    case 9: return reinterpret_cast<const void*>(gs_iterate<GS_LX, 9>);
    case 10: return reinterpret_cast<const void*>(gs_iterate<GS_LX, 10>);
    case 11: return reinterpret_cast<const void*>(gs_iterate<GS_LX, 11>);
    case 12: return reinterpret_cast<const void*>(gs_iterate<GS_LX, 12>);
    default: return nullptr;
  }
}

}  // namespace gsk
