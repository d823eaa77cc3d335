// gs_common.cuh -- pieces shared by the iteration kernels: pass kinds, the
// block's shared state, shared-memory offsets, error reporting, FP64 block
// and slot sums, and the bounded grid barrier.
#pragma once

#include <cstdint>

#include "gs.h"
#include "gs_internal.h"

namespace gsk {

enum PassKind { kInit = 0, kCol = 1, kRow = 2, kResid = 3, kInitM = 4 };

// A barrier wait gives up after this long and reports GS_ETIMEOUT.
constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;
constexpr unsigned kMaxSpins = 1u << 26;

struct Shared {
  uint64_t mbar;  // completion of the amplitude bulk copy
  int flag;
  int pending;    // a bulk copy into shared memory may still be in flight
  const float* m_block;  // global address of the amplitude block in shared memory (null: none)
  unsigned pending_phase;  // the mbarrier phase that copy completes
  // Column passes that keep two column blocks in flight, one per half of the
  // block (slot): each slot's completion mbarrier, resident amplitude block
  // and pending copy, as above.
  uint64_t mbar_s[2];
  const float* m_slot[2];
  int pend_s[2];
  unsigned pend_phase_s[2];
  double red[kThreads / 32];
  float redf[kThreads / 32];
  float scale[kMaxBatch];  // sqrt(N / sum I) per mask
  int bad[kMaxBatch];      // mask with a non-finite, negative or zero target
};

// Shared-memory layout of the iteration kernel (dynamic part): group exchange
// buffers, the staged amplitude columns, then the staged field columns.
constexpr int kAmpSmemBytes = 8192 * 4;  // amplitude of one column block (<= 8192 values)
constexpr int kAmpSmemOffset = kGroupSmemBytes;
constexpr int kBlockSmemOffset = kGroupSmemBytes + kAmpSmemBytes;
constexpr int kBlockSmemBytes = 8192 * 8;  // one column block of the field

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Added once to the grid-barrier counter by the first failing thread of a
// launch: it releases every waiting block, which sees the bit in the value its
// spin ended on (no extra load after the barrier). Arrivals per launch stay far
// below it (at most blocks x passes, < 2^20).
constexpr unsigned kAbortBit = 1u << 30;

__device__ __forceinline__ void fail(const Params& p, int code) {
  atomicCAS(p.status, 0, code);
  if (atomicExch(p.abort_flag, 1) == 0) atomicAdd(p.bar, kAbortBit);
}

// sum p^2 of the SLM amplitude (N for p = 1): the energy of every field in S.
__device__ __forceinline__ double energy_of(const Params& p) {
  return p.p_slm ? *p.energy : static_cast<double>(p.nx) * p.ny;
}

// Record an error for the host without stopping the run (other masks go on).
__device__ __forceinline__ void fail_status(const Params& p, int code) { atomicCAS(p.status, 0, code); }

// Contiguous share [lo, hi) of `total` items for block b of G.
__device__ __forceinline__ int split(int b, int G, int total) {
  return static_cast<int>((static_cast<long long>(b) * total) / G);
}

// Sum of one double per thread over the block, in a fixed order. The result
// is valid in thread 0 only (its one reader): FP64 issue is scarce on this
// part, so the sum of the warps' totals runs on one thread, not on all 256.
static __device__ double block_sum(double x, Shared& sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += sh.red[w];
  }
  return s;
}

// Sum of one float per thread over the block: FP32 within the block (warp
// shuffles, then the warps' totals on one thread), widened to FP64 for the
// grid-wide reduction, which runs in FP64 (warp_slot_sum). A warp's FP64
// shuffles would run on the FP64 pipe (1/64 of the FP32 rate on this part)
// and cost more than the pass's projection. The result is valid in thread 0.
static __device__ double block_sum_f(float x, Shared& sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh.redf[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t += sh.redf[w];
    s = static_cast<double>(t);
  }
  return s;
}

// Sum of partials[row][0..G) in a fixed order (row = slot * batch + mask),
// computed by one warp; the result is returned to every lane of that warp.
static __device__ double warp_slot_sum(const Params& p, int row) {
  const int G = gridDim.x;
  const double* src = p.partials + static_cast<size_t>(row) * G;
  double s = 0.0;
  for (int c = threadIdx.x & 31; c < G; c += 32) s += src[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Grid-wide barrier over a zero-initialised arrival counter. Returns false in
// every thread of the block if the wait gave up (status GS_ETIMEOUT).
static __device__ bool grid_sync(const Params& p, unsigned& target, Shared& sh) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    int ok = 1;
    // Arrival with release semantics at GPU scope: cumulative, so it covers
    // the block's writes that the __syncthreads above ordered before it
    // (bulk stores were completed and fenced by their issuing thread).
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p.bar) : "memory");
    const unsigned want = target + p.extra_arrivals;
    unsigned spins = 0;
    unsigned long long t0 = 0;
    unsigned v;
    while (static_cast<int>((v = ld_acquire_gpu(p.bar)) - want) < 0) {
      ++spins;
      if ((spins & 255u) == 0) {
        const unsigned long long now = global_ns();
        if (t0 == 0) t0 = now;
        if (now - t0 > kBarrierTimeoutNs || spins > kMaxSpins) {
          ok = 0;
          fail(p, GS_ETIMEOUT);
          break;
        }
      }
    }
    // The acquire load above orders this thread's later reads after every
    // block's arrival; the proxy fence extends that to the bulk copies it
    // issues next, and the __syncthreads below to the rest of the block.
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (ok && (v & kAbortBit) != 0) ok = 0;  // a block failed in this launch
    sh.flag = ok;
  }
  __syncthreads();
  return sh.flag != 0;
}

}  // namespace gsk
