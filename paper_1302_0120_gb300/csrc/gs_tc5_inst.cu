// gs_tc5_inst.cu -- the iteration kernel of 1024 x 1024 masks whose
// transforms run on the tensor cores through tcgen05 (FP16 or BF16 operands).
#include "gs_iterate.cuh"

namespace gsk {

const void* iterate_kernel_tc5(bool bf16) {
  return bf16 ? reinterpret_cast<const void*>(gs_iterate_tc5<true>) : reinterpret_cast<const void*>(gs_iterate_tc5<false>);
}

}  // namespace gsk
