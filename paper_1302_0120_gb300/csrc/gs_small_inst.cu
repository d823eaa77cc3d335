// gs_small_inst.cu -- the small-grid kernels (gs_small.cuh) for every grid of
// power-of-two sides >= 32 with at most kSmallMaxPixels pixels, and their
// host-side launch.
#include "gs_small.cuh"

namespace gsk {

namespace {

template <int LX, int LY>
struct SmallKernel {
  static const void* fn() { return reinterpret_cast<const void*>(&gs_small<LX, LY>); }
  static constexpr int kThreadsPerBlock = SmallGeom<LX, LY>::NT;
  static constexpr int kSmem = SmallGeom<LX, LY>::SMEM;
};

struct SmallEntry {
  const void* fn;
  int threads;
  int smem;
};

template <int LX, int LY>
SmallEntry entry() {
  return {SmallKernel<LX, LY>::fn(), SmallKernel<LX, LY>::kThreadsPerBlock, SmallKernel<LX, LY>::kSmem};
}

int log2_of(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

bool lookup(int nx, int ny, SmallEntry* e) {
  if (!small_grid(nx, ny)) return false;
  switch (log2_of(nx) * 16 + log2_of(ny)) {
    case 5 * 16 + 5: *e = entry<5, 5>(); return true;
    case 5 * 16 + 6: *e = entry<5, 6>(); return true;
    case 5 * 16 + 7: *e = entry<5, 7>(); return true;
    case 5 * 16 + 8: *e = entry<5, 8>(); return true;
    case 6 * 16 + 5: *e = entry<6, 5>(); return true;
    case 6 * 16 + 6: *e = entry<6, 6>(); return true;
    case 6 * 16 + 7: *e = entry<6, 7>(); return true;
    case 7 * 16 + 5: *e = entry<7, 5>(); return true;
    case 7 * 16 + 6: *e = entry<7, 6>(); return true;
    case 8 * 16 + 5: *e = entry<8, 5>(); return true;
    default: return false;
  }
}

}  // namespace

cudaError_t small_prepare(int nx, int ny) {
  SmallEntry e;
  if (!lookup(nx, ny, &e)) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, e.smem);
}

cudaError_t launch_small(const Params& p, cudaStream_t s) {
  SmallEntry e;
  if (!lookup(p.nx, p.ny, &e)) return cudaErrorInvalidValue;
  void* args[] = {const_cast<Params*>(&p)};
  return cudaLaunchKernel(e.fn, dim3(p.batch), dim3(e.threads), args, e.smem, s);
}

}  // namespace gsk
