// gs_small.cuh -- Gerchberg-Saxton on small grids: one block per mask, the
// whole run in shared memory.
//
// For grids of at most 8192 pixels (64 x 64, 32 x 256, 64 x 128, ...) the
// field (64 KiB at most) and the scaled amplitude fit in one block's shared
// memory, so a mask needs neither global round trips between passes nor grid
// barriers: one block runs A0 -> A1 -> (A2, A3) x K -> A4 of Eq. (e:AP) alone,
// with __syncthreads between passes, and a batch is one block per mask (two
// blocks per SM at 64 x 64). Each row and column is transformed by the same
// group FFT (gs_fft.cuh) and projected by the same arithmetic as in the
// persistent kernel (gs_iterate.cuh), so the iterates agree bit for bit; only
// the order of the FP64 gap sums differs.
//
// Shared-memory layout: the field F [ny][nx] with element (y, x) at
// y nx + (x ^ rev4(y)) (rev4: bit reversal of the low four bits of y), which
// keeps both the row accesses (T_x threads per row, rows of a half-warp at
// consecutive y) and the column accesses (T_y consecutive rows per column) of
// a half-warp on distinct 8-byte banks; the amplitude transposed, m[x][y] with
// row stride ny + T_y; then the groups' exchange buffers.
#pragma once

#include <cfloat>
#include <cmath>

#include "gs.h"
#include "gs_fft.cuh"
#include "gs_internal.h"

namespace gsk {

template <int LX, int LY>
struct SmallGeom {
  static constexpr int NX = 1 << LX;
  static constexpr int NY = 1 << LY;
  static constexpr int N = NX * NY;
  static constexpr int TX = NX >> 5;                     // threads per row transform
  static constexpr int TY = NY >> 5;                     // threads per column transform
  static constexpr int NT = (N / 32 < 256) ? N / 32 : 256;  // threads per block
  static constexpr int NGR = NT / TX;                    // rows per round
  static constexpr int NGC = NT / TY;                    // columns per round
  static constexpr int MLD = NY + TY;                    // row stride of the amplitude
  static constexpr int F_BYTES = N * 8;
  static constexpr int M_BYTES = (NX * MLD * 4 + 15) / 16 * 16;
  static constexpr int X_BYTES = NT * 33 * 8;            // (NT / T) groups of (n + n/32) complex
  static constexpr int SMEM = F_BYTES + M_BYTES + X_BYTES;
  static_assert(LX >= 5 && LY >= 5 && N <= kSmallMaxPixels, "small grids only");
  static_assert(NGR <= NY && NGC <= NX, "every group has a line in every round");
  __device__ static int rev4(int y) { return static_cast<int>(__brev(static_cast<unsigned>(y)) >> 28); }
  __device__ static int fo(int y, int x) { return y * NX + (x ^ rev4(y)); }
};

// Sum of one double per thread over a block of NT threads, in a fixed order.
template <int NT>
__device__ __forceinline__ double small_sum(double x, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();  // red is free
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) s += red[w];
  return s;
}

__device__ __forceinline__ float small_phase(float2 u) {
  const float ph = atan2f(u.y, u.x);
  return (ph <= -3.14159274f) ? 3.14159274f : ph;
}

enum SmallPass { kSmallInit = 0, kSmallRow = 1, kSmallCol = 2, kSmallResid = 3 };

// One pass over the rows (init, row) or columns (col, resid) of the block's
// mask; returns this thread's FP64 share of the pass's gap sum.
template <int LX, int LY, int KIND>
__device__ __forceinline__ double small_pass(const Params& p, size_t moff, bool last, float2* F, const float* mT,
                                             float2* X, const StageTw<LX>& twr, const StageTw<LY>& twc) {
  using Gm = SmallGeom<LX, LY>;
  constexpr bool kRows = (KIND == kSmallInit || KIND == kSmallRow);
  constexpr int LN = kRows ? LX : LY;
  constexpr int T = kRows ? Gm::TX : Gm::TY;
  constexpr int NG = kRows ? Gm::NGR : Gm::NGC;
  constexpr int LINES = kRows ? Gm::NY : Gm::NX;
  GroupT<LN> grp;
  grp.t = threadIdx.x & (T - 1);
  grp.bar_id = 0;  // T <= 8: groups sync by warp
  grp.sm = X + (threadIdx.x / T) * GroupT<LN>::SMEM;
  grp.tw = kRows ? p.twx : p.twy;
  const int t = grp.t;
  const float inv_sqrt_n = p.inv_sqrt_n;
  double acc = 0.0;
  const StageTw<LN>& stw = [&]() -> const StageTw<LN>& {
    if constexpr (kRows) return twr;
    else return twc;
  }();
  for (int l0 = 0; l0 < LINES; l0 += NG) {
    const int line = l0 + static_cast<int>(threadIdx.x) / T;
    float2 v[32];
    float part = 0.f;
    if constexpr (KIND == kSmallInit) {
      const float* ph = p.phi_in + moff + static_cast<size_t>(line) * Gm::NX + t;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        float s, c;
        sincosf(ph[T * i], &s, &c);
        v[i] = make_float2(c, s);  // u0 = exp(i phi0)
      }
      if (last) {  // zero iterations: the mask is arg exp(i phi0)
        float* po = p.phi_out + moff + static_cast<size_t>(line) * Gm::NX + t;
#pragma unroll
        for (int i = 0; i < 32; ++i) po[T * i] = small_phase(v[i]);
      }
      group_fft<LN>(v, grp, stw);
#pragma unroll
      for (int i = 0; i < 32; ++i) F[Gm::fo(line, t + T * i)] = v[i];
    } else if constexpr (KIND == kSmallRow) {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = F[Gm::fo(line, t + T * i)];
      // v = swap(IDFT_x(B)) = swap(sqrt(N) P_M u^nu): gap to S and Eq. (e:PS)
      group_fft<LN>(v, grp, stw);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float vx = v[i].y;
        const float vy = v[i].x;
        const float a2 = vx * vx + vy * vy;
        const float rs = rsqrtf(a2);
        const float mag = a2 > 0.f ? a2 * rs : 0.f;
        const float d = mag * inv_sqrt_n - 1.f;
        part += d * d;
        v[i] = a2 > 0.f ? make_float2(vx * rs, vy * rs) : make_float2(1.f, 0.f);
      }
      if (last) {
        float* po = p.phi_out + moff + static_cast<size_t>(line) * Gm::NX + t;
#pragma unroll
        for (int i = 0; i < 32; ++i) po[T * i] = small_phase(v[i]);
      }
      if (!last || p.final_resid) {
        group_fft<LN>(v, grp, stw);
#pragma unroll
        for (int i = 0; i < 32; ++i) F[Gm::fo(line, t + T * i)] = v[i];
      }
    } else {
      const int c = line;
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = F[Gm::fo(t + T * i, c)];
      // v = Y = F u^nu along this column: residual and Eq. (e:Mhat)
      group_fft<LN>(v, grp, stw);
      const float* mcol = mT + c * Gm::MLD + t;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float m = mcol[T * i];
        const float2 Y = v[i];
        const float a2 = Y.x * Y.x + Y.y * Y.y;
        const float rs = rsqrtf(a2);
        const float mag = a2 > 0.f ? a2 * rs : 0.f;
        const float d = mag * inv_sqrt_n - m;
        part += d * d;
        if constexpr (KIND == kSmallCol) {
          const float f = m * rs;
          const float2 Yh = a2 > 0.f ? make_float2(Y.x * f, Y.y * f) : make_float2(m, 0.f);
          v[i] = make_float2(Yh.y, Yh.x);  // swapped: the next forward DFT acts as the inverse
        }
      }
      if constexpr (KIND == kSmallCol) {
        group_fft<LN>(v, grp, stw);
#pragma unroll
        for (int i = 0; i < 32; ++i) F[Gm::fo(t + T * i, c)] = v[i];
      }
    }
    acc += static_cast<double>(part);
  }
  __syncthreads();  // the pass's writes are seen by the next pass
  return acc;
}

template <int LX, int LY>
__global__ void __launch_bounds__(SmallGeom<LX, LY>::NT) gs_small(const Params p) {
  using Gm = SmallGeom<LX, LY>;
  constexpr int NT = Gm::NT;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[NT / 32];
  float2* F = reinterpret_cast<float2*>(smem);
  float* mT = reinterpret_cast<float*>(smem + Gm::F_BYTES);
  float2* X = reinterpret_cast<float2*>(smem + Gm::F_BYTES + Gm::M_BYTES);
  const int mb = blockIdx.x;
  const size_t moff = static_cast<size_t>(mb) * static_cast<size_t>(p.mstride);
  const float* I = p.I + moff;
  double* r_out = p.r_out ? p.r_out + static_cast<size_t>(mb) * p.rstride : nullptr;
  double* g_out = p.g_out ? p.g_out + static_cast<size_t>(mb) * p.gstride : nullptr;
  const double energy = static_cast<double>(Gm::N);  // sum p^2 with p = 1

  // A0: sum I in FP64; a non-finite or negative pixel poisons it with NaN
  double acc = 0.0;
  bool bad = false;
  for (int e = threadIdx.x; e < Gm::N; e += NT) {
    const float x = I[e];
    bad |= !(x >= 0.f && x <= FLT_MAX);
    acc += static_cast<double>(x);
  }
  if (__syncthreads_or(bad)) acc = __longlong_as_double(0x7ff8000000000000ll);
  const double total = small_sum<NT>(acc, red);
  if (!(total > 0.0) || !(total <= DBL_MAX)) {
    // rejected: phase untouched, gaps NaN, GS_ENUMERIC
    if (threadIdx.x == 0) atomicCAS(p.status, 0, GS_ENUMERIC);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    if (r_out)
      for (int e = threadIdx.x; e < p.iters + (p.final_resid ? 1 : 0); e += NT) r_out[e] = nan;
    if (g_out)
      for (int e = threadIdx.x; e < p.iters; e += NT) g_out[e] = nan;
    return;
  }
  const float s = static_cast<float>(sqrt(energy / total));
  for (int e = threadIdx.x; e < Gm::N; e += NT) {
    const int y = e >> LX;
    const int x = e & (Gm::NX - 1);
    mT[x * Gm::MLD + y] = s * sqrtf(I[e]);
  }
  // stage twiddles of both lengths, held for the whole run
  StageTw<LX> twr;
  twr.load(p.twx, threadIdx.x & (Gm::TX - 1));
  StageTw<LY> twc;
  twc.load(p.twy, threadIdx.x & (Gm::TY - 1));
  __syncthreads();

  const int K = p.iters;
  small_pass<LX, LY, kSmallInit>(p, moff, K == 0, F, mT, X, twr, twc);
  for (int nu = 0; nu < K; ++nu) {
    const double rc = small_sum<NT>(small_pass<LX, LY, kSmallCol>(p, moff, false, F, mT, X, twr, twc), red);
    if (r_out && threadIdx.x == 0) r_out[nu] = sqrt(rc / energy);
    const double gr = small_sum<NT>(small_pass<LX, LY, kSmallRow>(p, moff, nu == K - 1, F, mT, X, twr, twc), red);
    if (g_out && threadIdx.x == 0) g_out[nu] = sqrt(gr / energy);
  }
  if (p.final_resid) {
    const double rc = small_sum<NT>(small_pass<LX, LY, kSmallResid>(p, moff, false, F, mT, X, twr, twc), red);
    if (r_out && threadIdx.x == 0) r_out[K] = sqrt(rc / energy);
  }
}

}  // namespace gsk
