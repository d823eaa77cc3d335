// gs_mixed_inst.cu -- the iteration kernel for batches of mixed square sizes
// (256, 512 and 1024 in one launch), FP32 and tensor-core forms.
#include "gs_iterate.cuh"

namespace gsk {

const void* iterate_kernel_mixed(bool tc) {
  return tc ? reinterpret_cast<const void*>(gs_iterate_mixed<true>)
            : reinterpret_cast<const void*>(gs_iterate_mixed<false>);
}

}  // namespace gsk
