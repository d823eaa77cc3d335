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

// Sum of one double per thread over a block of NT threads, in a fixed order,
// valid in thread 0 only (FP64 issue is scarce: one thread adds the warps'
// totals, not all of them).
template <int NT>
__device__ __forceinline__ double small_sum(double x, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();  // red is free
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += red[w];
  }
  return s;
}

// The same for one float per thread, in FP32 (the gaps of a pass: a warp's
// FP64 shuffles would run on the FP64 pipe, 1/64 of the FP32 rate here),
// widened to FP64 for the normalisation.
template <int NT>
__device__ __forceinline__ double small_sum_f(float x, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();  // red is free
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    s = static_cast<double>(t);
  }
  return s;
}

__device__ __forceinline__ float small_phase(float2 u) {
  const float ph = atan2f(u.y, u.x);
  return (ph <= -3.14159274f) ? 3.14159274f : ph;
}

// The phase of row `line` to phase_out, once per run: through the group's
// exchange buffer (free between transforms), so that a rolled loop holds the
// only copy of atan2f and the registers are never indexed at run time.
template <int LN>
__device__ __forceinline__ void small_phase_out(const Params& p, size_t moff, int line, int t, const float2 (&v)[32],
                                                const GroupT<LN>& grp) {
  constexpr int T = GroupT<LN>::T;
  float2* su = grp.sm + t;
#pragma unroll
  for (int i = 0; i < 32; ++i) su[T * i] = v[i];
  float* po = p.phi_out + moff + static_cast<size_t>(line) * GroupT<LN>::N + t;
#pragma unroll 1
  for (int i = 0; i < 32; ++i) po[T * i] = small_phase(su[T * i]);
  grp.sync();  // the next transform's exchange reuses the buffer
}

enum SmallPass { kSmallInit = 0, kSmallRow = 1, kSmallCol = 2, kSmallResid = 3 };

// The passes that run once per run: A1 (init, the rows of u0 = exp(i phi0))
// and A4's final residual (the columns, forward transform only). Returns this
// thread's FP64 share of the pass's gap sum.
template <int LX, int LY, int KIND>
__device__ __forceinline__ float small_pass(const Params& p, size_t moff, bool last, float2* F, const float* mT,
                                             float2* X, const StageTw<LX>& twr, const StageTw<LY>& twc) {
  static_assert(KIND == kSmallInit || KIND == kSmallResid, "the iteration passes are small_pass_hot");
  using Gm = SmallGeom<LX, LY>;
  constexpr bool kRows = (KIND == kSmallInit);
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
  float acc = 0.f;
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
      if (last) small_phase_out(p, moff, line, t, v, grp);  // zero iterations: arg exp(i phi0)
      group_fft<LN>(v, grp, stw);
#pragma unroll
      for (int i = 0; i < 32; ++i) F[Gm::fo(line, t + T * i)] = v[i];
    } else {
      const int c = line;
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = F[Gm::fo(t + T * i, c)];
      // v = Y = F u^K along this column: the final residual
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
      }
    }
    acc += part;
  }
  __syncthreads();  // the pass's writes are seen by the next pass
  return acc;
}

// The passes of the iteration loop, column (A2) or row (A3) by `kind` at run
// time, lines of length 2^LN. The two transforms of a line go through one
// rolled loop and a square grid serves both kinds with one instantiation, so
// the loop body holds a single copy of the unrolled FFT: with one warp per
// scheduler, a body with four copies spent most of its time waiting for
// instructions. ROWS / COLS: the kinds this instantiation serves.
template <int LX, int LY, int LN, bool ROWS, bool COLS>
__device__ __forceinline__ float small_pass_hot(const Params& p, size_t moff, int kind, bool last, float2* F,
                                                 const float* mT, float2* X, const StageTw<LN>& stw) {
  using Gm = SmallGeom<LX, LY>;
  static_assert(!ROWS || LN == LX, "row transforms have length nx");
  static_assert(!COLS || LN == LY, "column transforms have length ny");
  constexpr int T = 1 << (LN - 5);
  constexpr int NG = Gm::NT / T;
  constexpr int LINES = Gm::N >> LN;  // rows (length nx) or columns (length ny)
  const bool rows = ROWS && (!COLS || kind == kSmallRow);
  GroupT<LN> grp;
  grp.t = threadIdx.x & (T - 1);
  grp.bar_id = 0;  // T <= 8: groups sync by warp
  grp.sm = X + (threadIdx.x / T) * GroupT<LN>::SMEM;
  grp.tw = rows ? p.twx : p.twy;
  const int t = grp.t;
  const float inv_sqrt_n = p.inv_sqrt_n;
  // a row pass that ends the run without the final residual stops after the projection
  const int nh = (rows && last && !p.final_resid) ? 1 : 2;
  float acc = 0.f;
  for (int l0 = 0; l0 < LINES; l0 += NG) {
    const int line = l0 + static_cast<int>(threadIdx.x) / T;
    float2 v[32];
    float part = 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = F[rows ? Gm::fo(line, t + T * i) : Gm::fo(t + T * i, line)];
#pragma unroll 1
    for (int h = 0; h < nh; ++h) {
      group_fft<LN>(v, grp, stw);
      if (h != 0) continue;
      if (rows) {
        // v = swap(IDFT_x(B)) = swap(sqrt(N) P_M u^nu): gap to S and Eq. (e:PS)
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
        if (last) small_phase_out(p, moff, line, t, v, grp);
      } else {
        // v = Y = F u^nu along this column: residual and Eq. (e:Mhat)
        const float* mcol = mT + line * Gm::MLD + t;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float m = mcol[T * i];
          const float2 Y = v[i];
          const float a2 = Y.x * Y.x + Y.y * Y.y;
          const float rs = rsqrtf(a2);
          const float mag = a2 > 0.f ? a2 * rs : 0.f;
          const float d = mag * inv_sqrt_n - m;
          part += d * d;
          const float f = m * rs;
          const float2 Yh = a2 > 0.f ? make_float2(Y.x * f, Y.y * f) : make_float2(m, 0.f);
          v[i] = make_float2(Yh.y, Yh.x);  // swapped: the next forward DFT acts as the inverse
        }
      }
    }
    if (nh == 2) {
#pragma unroll
      for (int i = 0; i < 32; ++i) F[rows ? Gm::fo(line, t + T * i) : Gm::fo(t + T * i, line)] = v[i];
    }
    acc += part;
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
  __shared__ float redf[NT / 32];
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
  {
    const double t0 = small_sum<NT>(acc, red);
    if (threadIdx.x == 0) red[0] = t0;  // to every thread
    __syncthreads();
  }
  const double total = red[0];
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
  // pass q: column pass of iteration q/2 (q even), row pass (q odd)
#pragma unroll 1
  for (int q = 0; q < 2 * K; ++q) {
    const bool rows = (q & 1) != 0;
    const int nu = q >> 1;
    const bool last = rows && nu == K - 1;
    float a;
    if constexpr (LX == LY) {
      a = small_pass_hot<LX, LY, LX, true, true>(p, moff, rows ? kSmallRow : kSmallCol, last, F, mT, X, twr);
    } else {
      a = rows ? small_pass_hot<LX, LY, LX, true, false>(p, moff, kSmallRow, last, F, mT, X, twr)
               : small_pass_hot<LX, LY, LY, false, true>(p, moff, kSmallCol, false, F, mT, X, twc);
    }
    // the raw sum now, the normalisation after the loop (an FP64 division
    // and square root on one thread would hold up the next pass)
    const double sum = small_sum_f<NT>(a, redf);
    if (threadIdx.x == 0) {
      double* const out = rows ? g_out : r_out;
      if (out) out[nu] = sum;
    }
  }
  if (p.final_resid) {
    const double rc = small_sum_f<NT>(small_pass<LX, LY, kSmallResid>(p, moff, false, F, mT, X, twr, twc), redf);
    if (r_out && threadIdx.x == 0) r_out[K] = rc;
  }
  __syncthreads();  // thread 0's sums are visible to the block
  const int nr = K + (p.final_resid ? 1 : 0);
  if (r_out)
    for (int e = threadIdx.x; e < nr; e += NT) r_out[e] = sqrt(r_out[e] / energy);
  if (g_out)
    for (int e = threadIdx.x; e < K; e += NT) g_out[e] = sqrt(g_out[e] / energy);
}

}  // namespace gsk
