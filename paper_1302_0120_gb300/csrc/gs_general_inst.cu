// gs_general_inst.cu -- the iteration kernel for grids with a side that is
// not a power of two (gs_general.cuh).
#include "gs_iterate.cuh"

namespace gsk {

const void* iterate_kernel_general() { return reinterpret_cast<const void*>(gs_iterate<0, 0, false>); }

}  // namespace gsk
