// gs_tc5_inst.cu -- the iteration kernel of square 256, 512 and 1024 masks
// whose transforms run on the tensor cores through tcgen05 (FP16 or BF16
// operands).
#include "gs_iterate.cuh"

namespace gsk {

template <bool BF16>
static const void* tc5_for(int l) {
  switch (l) {
    case 8: return reinterpret_cast<const void*>(gs_iterate_tc5<8, BF16>);
    case 9: return reinterpret_cast<const void*>(gs_iterate_tc5<9, BF16>);
    case 10: return reinterpret_cast<const void*>(gs_iterate_tc5<10, BF16>);
    default: return nullptr;
  }
}

const void* iterate_kernel_tc5(int l, bool bf16) { return bf16 ? tc5_for<true>(l) : tc5_for<false>(l); }

}  // namespace gsk
