// gs_mixed_inst.cu -- the iteration kernel for batches of mixed square sizes
// (256, 512 and 1024 in one launch): FP32, mma.sync and tcgen05 forms.
#include "gs_iterate.cuh"

namespace gsk {

const void* iterate_kernel_mixed(int tc_mode) {
  switch (tc_mode) {
    case kTcMmaSync: return reinterpret_cast<const void*>(gs_iterate_mixed<true>);
    case kTcGen05F16: return reinterpret_cast<const void*>(gs_iterate_mixed_tc5<false>);
    case kTcGen05Bf16: return reinterpret_cast<const void*>(gs_iterate_mixed_tc5<true>);
    default: return reinterpret_cast<const void*>(gs_iterate_mixed<false>);
  }
}

}  // namespace gsk
