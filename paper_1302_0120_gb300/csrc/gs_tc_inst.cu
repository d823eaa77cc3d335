// gs_tc_inst.cu -- the iteration kernel with tensor-core transforms, for the
// square grids 256 x 256, 512 x 512 and 1024 x 1024.
#include "gs_iterate.cuh"

namespace gsk {

const void* iterate_kernel_tc(int l) {
  switch (l) {
    case 8: return reinterpret_cast<const void*>(gs_iterate<8, 8, true>);
    case 9: return reinterpret_cast<const void*>(gs_iterate<9, 9, true>);
    case 10: return reinterpret_cast<const void*>(gs_iterate<10, 10, true>);
    default: return nullptr;
  }
}

}  // namespace gsk
