// gs_rg.cuh -- register-resident passes for grids whose sides factor as
// n = T V with T, V <= 32 and are not both powers of two (600 = 24 x 25,
// 768 = 32 x 24, 800 = 32 x 25, 1024 = 32 x 32: the 800 x 600 SLM of Sec. V,
// the 1024 x 768 format). Other 5-smooth sides keep the shared-memory
// Stockham passes of gs_general.cuh.
//
// One warp holds one line (row or column) from load to store. A length-n
// transform is the four-step factorisation n = T V done by the warp:
//
//   layout (T, V): lane t < T holds x[t + T i], i < V
//   1. each lane: V-point DFT over i in registers (rdft<V>)
//   2. twiddle W_n^{t q}, q < V (table in shared memory, [q][t])
//   3. one exchange through the warp's padded shared-memory buffer
//   4. each lane q < V: T-point DFT over t in registers (rdft<T>)
//   layout (V, T): lane q < V holds X[q + V j], j < T
//
// since X[q + V j] = sum_t W_T^{t j} W_n^{t q} sum_i x[t + T i] W_V^{i q}. The
// output layout is the input layout with T and V exchanged, so the second
// transform of a pass (the inverse, by the swap identity of gs_fft.cuh) uses
// the factorisation (V, T) and returns the line to the layout (T, V) it was
// loaded in. Projections are elementwise and run in whichever layout the
// line is in; they, the gap sums and the pass schedule are those of the
// other kernels (gs_iterate.cuh).
//
// The field B is stored as in the power-of-two kernel: column blocks of 8
// adjacent columns, each one contiguous [ny][8] array whose rows are permuted
// by an XOR swizzle. A column pass moves a block (and its amplitude columns)
// with one bulk copy each way, one warp per column; a row pass reads and
// writes 64-byte row segments, one warp per row.
#pragma once

#include "gs_common.cuh"
#include "gs_general.cuh"
#include "gs_rg_dft.cuh"
#include "gs_tma.cuh"

namespace gsk {

// Factorisation n = T V of a length served here (T = threads of the first
// layout); rg_threads in gs_internal.h lists the lengths.
template <int N>
struct RgLen {
  static constexpr int T = rg_threads(N);
  static constexpr int V = N / (T > 0 ? T : 1);
  static_assert(T > 0 && T <= 32 && V <= 32 && T * V == N, "a length of the register-resident kernel");
  static constexpr int SA = T | 1;  // exchange row stride of the transform (T, V): odd, no bank conflicts
  static constexpr int SB = V | 1;  // ... of the transform (V, T)
  static constexpr int EX = (V * SA > T * SB) ? V * SA : T * SB;  // exchange entries
};

// Shared-memory layout of the register-resident kernel: twiddle tables of the
// row and column transforms (2 nx + 2 ny entries), one exchange buffer per
// warp, the amplitude of one column block, one column block of the field.
template <int NX, int NY>
struct RgSmem {
  static constexpr int kW = 8;  // columns per block
  static constexpr int EXW = ((RgLen<NX>::EX > RgLen<NY>::EX ? RgLen<NX>::EX : RgLen<NY>::EX) + 1) & ~1;
  static constexpr int kTw = 0;
  static constexpr int kEx = kTw + 2 * (NX + NY) * 8;
  static constexpr int kAmp = kEx + (kThreads / 32) * EXW * 8;
  static constexpr int kBlk = kAmp + ((kW * NY * 4 + 15) & ~15);
  static constexpr int kBytes = kBlk + kW * NY * 8;
  static_assert(kEx % 16 == 0 && kAmp % 16 == 0 && kBlk % 16 == 0, "bulk-copy destinations are 16-byte aligned");
  static_assert(kW * NY * 4 % 16 == 0, "bulk copies move multiples of 16 bytes");
};

// Storage of B: column blocks of 8 columns, [ny][8] each, XOR-swizzled rows.
template <int NX, int NY>
struct RgLayout {
  static constexpr int W = 8;
  static constexpr int BLOCK = NY * W;
  static_assert(NX % W == 0, "whole column blocks");
  __device__ static constexpr int swz(int y) { return (y >> 1) & (W - 1); }
  __device__ static size_t off(int y, int x) {
    return static_cast<size_t>(x >> 3) * BLOCK + y * W + ((x & (W - 1)) ^ swz(y));
  }
  __device__ static int boff(int y, int k) { return y * W + (k ^ swz(y)); }
};

// The twiddle tables, copied to shared memory once per launch. For a length
// n = T V the host writes n entries W_n^{t q} at [q T + t] (q < V, t < T) for
// the transform (T, V), then n entries W_n^{q j} at [j V + q] (j < T, q < V)
// for the transform (V, T).
template <int NX, int NY>
__device__ __forceinline__ void rg_load_twiddles(const Params& p, unsigned char* smem) {
  float2* t = reinterpret_cast<float2*>(smem + RgSmem<NX, NY>::kTw);
  for (int e = threadIdx.x; e < 2 * NX; e += kThreads) t[e] = p.twx[e];
  for (int e = threadIdx.x; e < 2 * NY; e += kThreads) t[2 * NX + e] = p.twy[e];
  __syncthreads();
}

// m = s sqrt(I), transposed ([nx][ny]) for the column passes, built by column
// blocks of 8 (this block's share): each block's [ny][8] slice of I is read in
// 32-byte row segments into a padded shared-memory tile, then written out
// column by column, both sides coalesced.
template <int NX, int NY>
__device__ __forceinline__ void rg_build_amplitude(const Params& p, int mb, float s, unsigned char* smem) {
  using L = RgLayout<NX, NY>;
  constexpr int W = L::W;
  static_assert(NY * (W + 1) * 4 <= W * NY * 8, "the tile fits the field block buffer");
  const size_t moff = static_cast<size_t>(mb) * static_cast<size_t>(p.mstride);
  const float* const Im = p.I + moff;
  float* const mTm = p.mT + moff;
  float* const tile = reinterpret_cast<float*>(smem + RgSmem<NX, NY>::kBlk);
  const int lo = split(blockIdx.x, gridDim.x, NX / W);
  const int hi = split(blockIdx.x + 1, gridDim.x, NX / W);
  for (int cb = lo; cb < hi; ++cb) {
    __syncthreads();
    for (int e = threadIdx.x; e < NY * W; e += kThreads) {
      const int y = e / W, k = e % W;
      tile[y * (W + 1) + k] = Im[static_cast<size_t>(y) * NX + cb * W + k];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < W * NY; e += kThreads) {
      const int k = e / NY, y = e % NY;
      mTm[static_cast<size_t>(cb * W + k) * NY + y] = s * sqrtf(tile[y * (W + 1) + k]);
    }
  }
  __syncthreads();
}

// The transform of a length-n line (n = T V) by one warp, layout (T, V) in,
// layout (V, T) out (see the top of this file). x has room for both layouts;
// lanes outside the active range compute on whatever they hold and write
// nothing. `tw` is the table of this factorisation, `ex` the warp's buffer.
template <int T, int V, int M>
__device__ __forceinline__ void rg_warp_dft(float2 (&x)[M], float2* __restrict__ ex, const float2* __restrict__ tw,
                                            int lane) {
  static_assert(M >= T && M >= V, "the line fits the register array");
  constexpr int S = T | 1;
  float2 a[V];
#pragma unroll
  for (int i = 0; i < V; ++i) a[i] = x[i];
  rdft<V>(a);
  const int tl = lane < T ? lane : 0;
#pragma unroll
  for (int q = 1; q < V; ++q) a[q] = cmul(a[q], tw[q * T + tl]);
  if (lane < T) {
#pragma unroll
    for (int q = 0; q < V; ++q) ex[q * S + lane] = a[q];
  }
  __syncwarp();
  float2 b[T];
  const int ql = lane < V ? lane : 0;
#pragma unroll
  for (int t = 0; t < T; ++t) b[t] = ex[ql * S + t];
  __syncwarp();  // the buffer is free for the next exchange
  rdft<T>(b);
#pragma unroll
  for (int j = 0; j < T; ++j) x[j] = b[j];
}

// Wrap an angle as the other kernels do: (-pi, pi].
__device__ __forceinline__ float rg_phase(float2 u) {
  const float a = atan2f(u.y, u.x);
  return (a <= -3.14159274f) ? 3.14159274f : a;
}

// One pass over rows [lo, hi) (kInit, kRow) or column blocks [lo, hi) (kCol,
// kResid, kInitM) of mask mb; the arithmetic of each kind is that of
// run_pass (gs_iterate.cuh). Returns this thread's share of the pass's gap sum.
template <int NX, int NY>
__device__ __forceinline__ float run_pass_rg(const Params& p, int mb, int kind, bool last, int lo, int hi,
                                             unsigned char* smem, Shared& sh, unsigned& mphase) {
  using SM = RgSmem<NX, NY>;
  using L = RgLayout<NX, NY>;
  using RX = RgLen<NX>;
  using RY = RgLen<NY>;
  constexpr int M = 32;
  const size_t moff = static_cast<size_t>(mb) * static_cast<size_t>(p.mstride);
  float2* const Bm = p.B + moff;
  const float* const mTm = p.mT + moff;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const float2* const tw = reinterpret_cast<const float2*>(smem + SM::kTw);
  float2* const ex = reinterpret_cast<float2*>(smem + SM::kEx) + warp * SM::EXW;
  const float inv_sqrt_n = p.inv_sqrt_n;
  const bool two = (kind == kCol || (kind == kRow && !(last && !p.final_resid)));
  float acc = 0.f;

  if (kind == kInit || kind == kRow) {
    constexpr int T = RX::T, V = RX::V;
    const float2* const twA = tw;       // (T, V)
    const float2* const twB = tw + NX;  // (V, T)
    for (int base = lo; base < hi; base += kThreads / 32) {
      const int idx = base + warp;
      const bool valid = idx < hi;
      const int ridx = valid ? idx : base;  // warps past the end work on a valid copy and store nothing
      const int tl = lane < T ? lane : 0;
      float2 v[M];
      if (kind == kInit) {
        // u0 = p exp(i phi0), once per run: a rolled loop through the warp's
        // exchange buffer (element order) keeps a single copy of sincosf and
        // atan2f in the kernel
        const float* ph = p.phi_in + moff + static_cast<size_t>(ridx) * NX;
        const float* pp = p.p_slm ? p.p_slm + static_cast<size_t>(ridx) * NX : nullptr;
#pragma unroll 1
        for (int e = lane; e < NX; e += 32) {
          float s, c;
          sincosf(ph[e], &s, &c);
          const float a = pp ? pp[e] : 1.f;
          ex[e] = make_float2(a * c, a * s);
        }
        if (last && valid) {  // zero iterations: the mask is arg exp(i phi^0)
          float* po = p.phi_out + moff + static_cast<size_t>(idx) * NX;
#pragma unroll 1
          for (int e = lane; e < NX; e += 32) po[e] = rg_phase(ex[e]);
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < V; ++i) v[i] = ex[tl + T * i];  // layout (T, V)
        __syncwarp();
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i) v[i] = Bm[L::off(ridx, tl + T * i)];
      }
      rg_warp_dft<T, V>(v, ex, twA, lane);  // now layout (V, T): lane q holds element q + V j
      float part = 0.f;
      if (kind == kRow) {
        // v = swap(IDFT_x(B)) = swap(sqrt(N) P_M u^nu). Gap to S and Eq. (e:PS).
        const int ql = lane < V ? lane : 0;
        const float* pp = p.p_slm ? p.p_slm + static_cast<size_t>(ridx) * NX + ql : nullptr;
#pragma unroll
        for (int j = 0; j < T; ++j) {
          const float a = pp ? pp[V * j] : 1.f;
          const float vx = v[j].y;
          const float vy = v[j].x;
          const float a2 = vx * vx + vy * vy;
          const float rs = rsqrtf(a2);
          const float mag = a2 > 0.f ? a2 * rs : 0.f;
          const float d = mag * inv_sqrt_n - a;
          part += d * d;
          const float f = a * rs;
          v[j] = a2 > 0.f ? make_float2(vx * f, vy * f) : make_float2(a, 0.f);
        }
        if (lane >= V) part = 0.f;
        if (last) {  // the mask, once per run, through the exchange buffer (element order)
          if (lane < V) {
#pragma unroll
            for (int j = 0; j < T; ++j) ex[lane + V * j] = v[j];
          }
          __syncwarp();
          if (valid) {
            float* po = p.phi_out + moff + static_cast<size_t>(idx) * NX;
#pragma unroll 1
            for (int e = lane; e < NX; e += 32) po[e] = rg_phase(ex[e]);
          }
          __syncwarp();
        }
        if (two) {
          rg_warp_dft<V, T>(v, ex, twB, lane);  // back to layout (T, V)
          if (valid && lane < T) {
#pragma unroll
            for (int i = 0; i < V; ++i) Bm[L::off(idx, lane + T * i)] = v[i];
          }
        }
      } else if (valid && lane < V) {  // kInit: B = DFT_x(u0), stored from layout (V, T)
#pragma unroll
        for (int j = 0; j < T; ++j) Bm[L::off(idx, lane + V * j)] = v[j];
      }
      if (valid) acc += part;
    }
    return acc;
  }

  // Column passes: one column block (8 columns) per round, one warp per column.
  constexpr int T = RY::T, V = RY::V;
  const float2* const twA = tw + 2 * NX;       // (T, V)
  const float2* const twB = tw + 2 * NX + NY;  // (V, T)
  float* const ms = reinterpret_cast<float*>(smem + SM::kAmp);
  float2* const blk = reinterpret_cast<float2*>(smem + SM::kBlk);
  const bool from_m = (kind == kInitM);  // transform m itself (the target start)
  const bool store = (kind == kCol || from_m);
  for (int cb = lo; cb < hi; ++cb) {
    __syncthreads();  // the previous round is done with the staging buffers
    if (threadIdx.x == 0) {
      bulk_wait_read_all();  // a previous bulk store has read blk
      fence_proxy_async_smem();
      const float* const msrc = mTm + static_cast<size_t>(cb) * L::BLOCK;
      const bool need_m = (sh.m_block != msrc);
      const unsigned bytes_b = from_m ? 0u : L::BLOCK * 8u;
      const unsigned bytes_m = L::BLOCK * 4u;
      mbar_arrive_expect_tx(&sh.mbar, bytes_b + (need_m ? bytes_m : 0u));
      if (!from_m) bulk_g2s(blk, Bm + static_cast<size_t>(cb) * L::BLOCK, bytes_b, &sh.mbar);
      // columns 8 cb .. 8 cb + 7 of m are contiguous in the transposed amplitude
      if (need_m) bulk_g2s(ms, msrc, bytes_m, &sh.mbar);
      sh.m_block = msrc;
      sh.pending = 1;
      sh.pending_phase = mphase & 1u;
    }
    const bool landed = mbar_wait_bounded(&sh.mbar, mphase & 1u);
    mphase ^= 1u;
    if (!landed) {
      fail(p, GS_ETIMEOUT);
    } else if (threadIdx.x == 0) {
      sh.pending = 0;
    }
    if (from_m) {
      // stage swap((m, 0)), so that the forward DFT below yields swap(IDFT_y(m))
      for (int e = threadIdx.x; e < L::BLOCK; e += kThreads) {
        const int k = e % L::W;
        const int y = e / L::W;
        blk[L::boff(y, k)] = make_float2(0.f, ms[k * NY + y]);
      }
      __syncthreads();
    }
    const int tl = lane < T ? lane : 0;
    float2 v[M];
#pragma unroll
    for (int i = 0; i < V; ++i) v[i] = blk[L::boff(tl + T * i, warp)];
    rg_warp_dft<T, V>(v, ex, twA, lane);  // layout (V, T)
    if (!from_m) {
      // v = Y = F u^nu along this column. Residual and Eq. (e:Mhat).
      const int ql = lane < V ? lane : 0;
      const float* mcol = ms + warp * NY + ql;
      float part = 0.f;
#pragma unroll
      for (int j = 0; j < T; ++j) {
        const float m = mcol[V * j];
        const float2 Y = v[j];
        const float a2 = Y.x * Y.x + Y.y * Y.y;
        const float rs = rsqrtf(a2);
        const float mag = a2 > 0.f ? a2 * rs : 0.f;
        const float d = mag * inv_sqrt_n - m;
        part += d * d;
        if (kind == kCol) {
          const float f = m * rs;
          const float2 Yh = a2 > 0.f ? make_float2(Y.x * f, Y.y * f) : make_float2(m, 0.f);
          v[j] = make_float2(Yh.y, Yh.x);  // swapped: the next forward DFT acts as the inverse
        }
      }
      if (lane < V) acc += part;
    }
    if (kind == kCol) {
      rg_warp_dft<V, T>(v, ex, twB, lane);  // back to layout (T, V)
      if (lane < T) {
#pragma unroll
        for (int i = 0; i < V; ++i) blk[L::boff(lane + T * i, warp)] = v[i];
      }
    } else if (from_m && lane < V) {  // one transform: stored from layout (V, T)
#pragma unroll
      for (int j = 0; j < T; ++j) blk[L::boff(lane + V * j, warp)] = v[j];
    }
    if (store) {
      __syncthreads();
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        bulk_s2g(Bm + static_cast<size_t>(cb) * L::BLOCK, blk, L::BLOCK * 8u);
        bulk_commit();
      }
    }
  }
  // the field must be in global memory before the grid barrier releases the next pass
  if (store && threadIdx.x == 0) bulk_wait_all();
  return acc;
}

}  // namespace gsk
