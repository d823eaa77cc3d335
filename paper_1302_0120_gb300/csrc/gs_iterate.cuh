// gs_iterate.cuh -- the persistent Gerchberg-Saxton iteration kernel for sm_103a.
//
// The kernel is a template on (log2 nx, log2 ny); gs_inst.cu instantiates it.
//
// One cooperative launch runs a whole run (or a chunk of up to 128 iterations)
// of Eq. (e:AP), u^{nu+1} = P_S P_M u^nu, as a sequence of passes over the
// field separated by grid barriers:
//
//   A0  sum of I (FP64) -> m = sqrt(I) sqrt(N / sum I), stored transposed
//       (Eq. pattern-constraint: m is the OSP amplitude)
//   A1  init rows:   u^0 = exp(i phi^0), B = DFT_x(u^0)
//   per iteration nu:
//   A2  column pass: Y = DFT_y(B) = F u^nu; r^nu from | |Y|/sqrt(N) - m |;
//                    Yhat = m Y/|Y| (Eq. e:Mhat); B = IDFT_y(Yhat)
//   A3  row pass:    v = IDFT_x(B) = sqrt(N) P_M u^nu (Eq. e:PM); g^nu from
//                    | |v|/sqrt(N) - 1 |; u = v/|v| (Eq. e:PS); B = DFT_x(u)
//                    (the last one writes phi = arg u instead, and B too when
//                    the final residual is requested)
//   A4  column pass, forward only: r^K.
//
// Each pass keeps a row (or column) in the registers of one thread group
// (gs_fft.cuh) from the moment it is loaded to the moment it is stored, so one
// iteration reads and writes the field exactly twice. Columns are staged
// through shared memory so that global accesses stay coalesced. Only forward
// transforms are issued: the inverse transforms are obtained by swapping
// real and imaginary parts, which is folded into the projections, so B holds
// swap(IDFT_y(Yhat)) between a column pass and the next row pass.
//
// FP64 is used only for the per-block partial sums of the target energy and
// of the two gaps; the field is FP32.
#pragma once

#include <cfloat>
#include <cmath>

#include "gs.h"
#include "gs_fft.cuh"
#include "gs_internal.h"
#include "gs_tma.cuh"

namespace gsk {

enum PassKind { kInit = 0, kCol = 1, kRow = 2, kResid = 3 };

// A barrier wait gives up after this long and reports GS_ETIMEOUT.
constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;
constexpr unsigned kMaxSpins = 1u << 26;

struct Shared {
  uint64_t mbar;  // completion of the amplitude bulk copy
  int flag;
  int pending;    // a bulk copy into shared memory may still be in flight
  unsigned pending_phase;  // the mbarrier phase that copy completes
  double red[kThreads / 32];
};

// Shared-memory layout of the iteration kernel (dynamic part): group exchange
// buffers, the staged amplitude columns, then the staged field columns.
constexpr int kAmpSmemBytes = 8192 * 4;  // W columns x N rows of m, W N = 8192
constexpr int kAmpSmemOffset = kGroupSmemBytes;
constexpr int kBlockSmemOffset = kGroupSmemBytes + kAmpSmemBytes;

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

__device__ __forceinline__ void fail(const Params& p, int code) {
  atomicCAS(p.status, 0, code);
  atomicExch(p.abort_flag, 1);
}

// Contiguous share [lo, hi) of `total` items for block b of G.
__device__ __forceinline__ int split(int b, int G, int total) {
  return static_cast<int>((static_cast<long long>(b) * total) / G);
}

// Sum of one double per thread over the block, in a fixed order. The result
// is returned to every thread.
static __device__ double block_sum(double x, Shared& sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) s += sh.red[w];
  return s;
}

// Sum of partials[slot][0..G) in a fixed order, computed by one warp; the
// result is returned to every lane of that warp.
static __device__ double warp_slot_sum(const Params& p, int slot) {
  const int G = gridDim.x;
  const double* src = p.partials + static_cast<size_t>(slot) * G;
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
    __threadfence();
    atomicAdd(p.bar, 1u);
    const unsigned want = target + p.extra_arrivals;
    unsigned spins = 0;
    unsigned long long t0 = 0;
    while (static_cast<int>(ld_acquire_gpu(p.bar) - want) < 0) {
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
    __threadfence();
    if (ok && *reinterpret_cast<volatile int*>(p.abort_flag) != 0) ok = 0;  // another block failed
    sh.flag = ok;
  }
  __syncthreads();
  return sh.flag != 0;
}

// One pass over this block's share of rows (kInit, kRow; LOGN = log2 nx) or
// columns (kCol, kResid; LOGN = log2 ny); LX = log2 nx. Returns this thread's
// FP64 contribution to the pass's gap sum.
template <int LOGN, int LX>
__device__ __forceinline__ double run_pass(const Params& p, int kind, bool last, unsigned char* smem, Shared& sh,
                                           unsigned& mphase) {
  using G = GroupT<LOGN>;
  constexpr int N = G::N;
  constexpr int T = G::T;
  constexpr int NX = 1 << LX;
  constexpr int LOGT = LOGN - 5;
  constexpr int LOGNG = 8 - LOGT;  // log2(kThreads / T)
  constexpr int NG = 1 << LOGNG;   // groups per block
  constexpr int W = NG;            // columns per staged block
  constexpr int WS = W + 1;        // padded row stride of the staged block
  constexpr int RSTEP = kThreads / W;  // block rows one sweep of the threads covers
  static_assert(kThreads == 256, "geometry assumes 256 threads");
  static_assert(N * W == 8192, "a staged block holds 8192 elements");
  const bool rows = (kind == kInit || kind == kRow);
  const int g = threadIdx.x >> LOGT;
  G grp;
  grp.t = threadIdx.x & (T - 1);
  grp.bar_id = 1 + g;
  grp.sm = reinterpret_cast<float2*>(smem) + g * G::SMEM;
  grp.tw = rows ? p.twx : p.twy;
  const int t = grp.t;
  float* ms = reinterpret_cast<float*>(smem + kAmpSmemOffset);
  float2* blk = reinterpret_cast<float2*>(smem + kBlockSmemOffset);
  const int total = rows ? p.ny : NX;
  const int lo = split(blockIdx.x, gridDim.x, total);
  const int hi = split(blockIdx.x + 1, gridDim.x, total);
  const int nfft = (kind == kCol || (kind == kRow && !(last && !p.final_resid))) ? 2 : 1;
  const float inv_sqrt_n = p.inv_sqrt_n;
  double acc = 0.0;

  for (int base = lo; base < hi; base += NG) {
    const int idx = base + g;
    const bool valid = idx < hi;
    const int ridx = valid ? idx : base;  // groups past the end work on a valid copy and store nothing
    const int wcur = min(NG, hi - base);
    float2 v[32];
    if (kind == kInit) {
      const float* ph = p.phi_in + static_cast<size_t>(ridx) * N + t;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        float s, c;
        sincosf(ph[T * i], &s, &c);
        v[i] = make_float2(c, s);
      }
      if (last && valid) {  // zero iterations: the mask is arg exp(i phi^0)
        float* po = p.phi_out + static_cast<size_t>(idx) * N + t;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float ph_out = atan2f(v[i].y, v[i].x);
          po[T * i] = (ph_out <= -3.14159274f) ? 3.14159274f : ph_out;
        }
      }
    } else if (kind == kRow) {
      const float2* src = p.B + static_cast<size_t>(ridx) * N + t;
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = src[T * i];
    } else {
      __syncthreads();  // previous round's readers of the staging buffers are done
      if (threadIdx.x == 0) {
        // Columns [base, base + wcur) of m are contiguous in the transposed
        // amplitude: one bulk copy, completed on the block's mbarrier.
        const unsigned bytes = static_cast<unsigned>(wcur) * N * 4u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&sh.mbar, bytes);
        bulk_g2s(ms, p.mT + static_cast<size_t>(base) * N, bytes, &sh.mbar);
        sh.pending = 1;
        sh.pending_phase = mphase;
      }
      // Stage columns [base, base + wcur) of B (N rows) through shared memory.
      const int k = threadIdx.x & (W - 1);
      const int y0 = threadIdx.x >> LOGNG;
      if (k < wcur) {
        const float2* src = p.B + static_cast<size_t>(y0) * NX + base + k;
        float2* dst = blk + y0 * WS + k;
#pragma unroll 8
        for (int j = 0; j < N / RSTEP; ++j) dst[j * RSTEP * WS] = src[static_cast<size_t>(j) * RSTEP * NX];
      }
      __syncthreads();
      const float2* src = blk + t * WS + g;
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = src[i * T * WS];
    }

    float part = 0.f;
#pragma unroll 1
    for (int h = 0; h < nfft; ++h) {
      group_fft<LOGN>(v, grp);
      if (h != 0) continue;
      if (kind == kCol || kind == kResid) {
        // v = Y = F u^nu along this column. Residual and Eq. (e:Mhat).
        if (!mbar_wait_bounded(&sh.mbar, mphase)) {
          fail(p, GS_ETIMEOUT);
        } else if (threadIdx.x == 0) {
          sh.pending = 0;
        }
        mphase ^= 1u;
        const float* mcol = ms + g * N + t;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float m = mcol[T * i];
          const float2 Y = v[i];
          const float a2 = Y.x * Y.x + Y.y * Y.y;
          const float rs = rsqrtf(a2);
          const float mag = a2 > 0.f ? a2 * rs : 0.f;
          const float d = mag * inv_sqrt_n - m;
          part += d * d;
          if (kind == kCol) {
            const float f = m * rs;
            const float2 Yh = a2 > 0.f ? make_float2(Y.x * f, Y.y * f) : make_float2(m, 0.f);
            v[i] = make_float2(Yh.y, Yh.x);  // swapped: the next forward DFT acts as the inverse
          }
        }
      } else if (kind == kRow) {
        // v = swap(IDFT_x(B)) = swap(sqrt(N) P_M u^nu). Gap to S and Eq. (e:PS).
        float* po = p.phi_out + static_cast<size_t>(ridx) * N + t;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float vx = v[i].y;
          const float vy = v[i].x;
          const float a2 = vx * vx + vy * vy;
          const float rs = rsqrtf(a2);
          const float mag = a2 > 0.f ? a2 * rs : 0.f;
          const float d = mag * inv_sqrt_n - 1.f;
          part += d * d;
          const float2 u = a2 > 0.f ? make_float2(vx * rs, vy * rs) : make_float2(1.f, 0.f);
          if (last && valid) {
            const float ph_out = atan2f(u.y, u.x);
            po[T * i] = (ph_out <= -3.14159274f) ? 3.14159274f : ph_out;
          }
          v[i] = u;
        }
      }
    }
    if (valid) acc += static_cast<double>(part);

    if (kind == kInit || (kind == kRow && nfft == 2)) {
      if (valid) {
        float2* dst = p.B + static_cast<size_t>(idx) * N + t;
#pragma unroll
        for (int i = 0; i < 32; ++i) dst[T * i] = v[i];
      }
    } else if (kind == kCol) {
      float2* dstb = blk + t * WS + g;
#pragma unroll
      for (int i = 0; i < 32; ++i) dstb[i * T * WS] = v[i];
      __syncthreads();
      const int k = threadIdx.x & (W - 1);
      const int y0 = threadIdx.x >> LOGNG;
      if (k < wcur) {
        float2* dst = p.B + static_cast<size_t>(y0) * NX + base + k;
        const float2* srcb = blk + y0 * WS + k;
#pragma unroll 8
        for (int j = 0; j < N / RSTEP; ++j) dst[static_cast<size_t>(j) * RSTEP * NX] = srcb[j * RSTEP * WS];
      }
    }
  }
  return acc;
}

// Before leaving after a failure, give a bulk copy that may still target this
// block's shared memory a bounded time to land.
static __device__ void drain_copies(Shared& sh) {
  if (threadIdx.x == 0 && sh.pending) mbar_wait_bounded(&sh.mbar, sh.pending_phase);
  __syncthreads();
}

// m = s sqrt(I) for this block's columns, written transposed ([nx][ny]) so
// that the column pass reads it contiguously.
static __device__ void build_amplitude(const Params& p, float s, unsigned char* smem) {
  const int logNG = 8 - (p.logny - 5);
  const int W = 1 << logNG;
  float* blk = reinterpret_cast<float*>(smem + kBlockSmemOffset);
  const int lo = split(blockIdx.x, gridDim.x, p.nx);
  const int hi = split(blockIdx.x + 1, gridDim.x, p.nx);
  for (int base = lo; base < hi; base += W) {
    const int wcur = min(W, hi - base);
    __syncthreads();
    for (int e = threadIdx.x; e < p.ny * W; e += kThreads) {
      const int k = e & (W - 1);
      const int y = e >> logNG;
      if (k < wcur) blk[y * (W + 1) + k] = p.I[static_cast<size_t>(y) * p.nx + base + k];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < wcur * p.ny; e += kThreads) {
      const int k = e >> p.logny;
      const int y = e & (p.ny - 1);
      p.mT[static_cast<size_t>(base + k) * p.ny + y] = s * sqrtf(blk[y * (W + 1) + k]);
    }
  }
  __syncthreads();
}

template <int LX, int LY>
__global__ void __launch_bounds__(kThreads, 1) gs_iterate(const Params p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shared sh;
  if (*reinterpret_cast<volatile int*>(p.abort_flag) != 0) return;  // an earlier chunk failed
  const int G = gridDim.x;
  const int b = blockIdx.x;
  unsigned target = 0;
  unsigned mphase = 0;
  if (threadIdx.x == 0) {
    mbar_init(&sh.mbar, 1);
    fence_barrier_init();
    sh.pending = 0;
  }
  __syncthreads();

  if (p.do_init) {
    // A0: FP64 energy of the target over this block's rows. A non-finite or
    // negative pixel poisons the sum with NaN.
    const int r0 = split(b, G, p.ny);
    const int r1 = split(b + 1, G, p.ny);
    const float* I = p.I + static_cast<size_t>(r0) * p.nx;
    const int cnt = (r1 - r0) * p.nx;
    double acc = 0.0;
    bool bad = false;
    for (int e = threadIdx.x; e < cnt; e += kThreads) {
      const float x = I[e];
      bad |= !(x >= 0.f && x <= FLT_MAX);
      acc += static_cast<double>(x);
    }
    if (bad) acc = __longlong_as_double(0x7ff8000000000000ll);
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) p.partials[b] = tot;
    if (!grid_sync(p, target, sh)) return;
    if (threadIdx.x < 32) {
      const double total = warp_slot_sum(p, 0);
      if (threadIdx.x == 0) sh.red[0] = total;
    }
    __syncthreads();
    const double total = sh.red[0];
    if (!(total > 0.0) || !(total <= DBL_MAX)) {
      if (b == 0) {
        if (threadIdx.x == 0) fail(p, GS_ENUMERIC);
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        const int nr = p.iters + (p.final_resid ? 1 : 0);
        if (p.r_out)
          for (int e = threadIdx.x; e < nr; e += kThreads) p.r_out[e] = nan;
        if (p.g_out)
          for (int e = threadIdx.x; e < p.iters; e += kThreads) p.g_out[e] = nan;
      }
      return;
    }
    const float s = static_cast<float>(sqrt(static_cast<double>(p.nx) * p.ny / total));
    build_amplitude(p, s, smem);
  }

  // Pass schedule: [init] (col, row) x nit [resid]. Slot of pass q (after
  // init) is 1 + q.
  const int nit = p.it1 - p.it0;
  const int resid = (p.do_final && p.final_resid) ? 1 : 0;
  const int npass = p.do_init + 2 * nit + resid;
  for (int q0 = 0; q0 < npass; ++q0) {
    int kind;
    int slot = -1;
    bool last = false;
    const int q = q0 - p.do_init;
    if (q < 0) {
      kind = kInit;
      last = p.do_final && p.iters == 0;
    } else if (q < 2 * nit) {
      kind = (q & 1) ? kRow : kCol;
      slot = 1 + q;
      last = (kind == kRow) && p.do_final && (p.it0 + (q >> 1) == p.iters - 1);
    } else {
      kind = kResid;
      slot = 1 + q;
    }
    double a;
    if constexpr (LX == LY) {
      a = run_pass<LX, LX>(p, kind, last, smem, sh, mphase);
    } else {
      a = (kind == kInit || kind == kRow) ? run_pass<LX, LX>(p, kind, last, smem, sh, mphase)
                                          : run_pass<LY, LX>(p, kind, last, smem, sh, mphase);
    }
    if (slot >= 0) {
      const double tot = block_sum(a, sh);
      if (threadIdx.x == 0) p.partials[static_cast<size_t>(slot) * G + b] = tot;
    }
    if (!grid_sync(p, target, sh)) {
      drain_copies(sh);
      return;
    }
  }

  // Gaps: r from column passes, g from row passes, in FP64.
  const int nslots = 2 * nit + resid;
  if (threadIdx.x < 32) {
    for (int s = 1 + b; s <= nslots; s += G) {
      const double sum = warp_slot_sum(p, s);
      if (threadIdx.x == 0) {
        const double val = sqrt(sum * p.inv_n);
        const int q = s - 1;
        if (q < 2 * nit) {
          const int nu = p.it0 + (q >> 1);
          if ((q & 1) == 0) {
            if (p.r_out) p.r_out[nu] = val;
          } else {
            if (p.g_out) p.g_out[nu] = val;
          }
        } else if (p.r_out) {
          p.r_out[p.iters] = val;
        }
      }
    }
  }
}

}  // namespace gsk
