// gs_iterate.cuh -- the persistent Gerchberg-Saxton iteration kernel for sm_103a.
//
// The kernel is a template on (log2 nx, log2 ny) and on where the transforms
// run: the FP32 ALUs (gs_fft.cuh; gs_inst.cu instantiates every size) or the
// tensor cores (gs_tc.cuh; gs_tc_inst.cu, square 256, 512 and 1024).
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
#include <type_traits>

#include "gs.h"
#include "gs_common.cuh"
#include "gs_fft.cuh"
#include "gs_general.cuh"
#include "gs_rg.cuh"
#include "gs_internal.h"
#include "gs_tc.cuh"
#include "gs_tc5.cuh"
#include "gs_tma.cuh"

namespace gsk {

// Tensor-core kernels only: the block's stage twiddles and cos/sin table.
constexpr int kTcTwOffset = kBlockSmemOffset + kBlockSmemBytes;
constexpr int kTcCsOffset = kTcTwOffset + kTcTwBytes;
static_assert(kTcTwBytes + kTcCsBytes == kTcExtraSmemBytes, "tensor-core tables match the launch size");

// Stands in for TcFft in the kernels whose transforms run on the FP32 ALUs.
struct NoTc {
  static constexpr bool kEnabled = false;
  static constexpr bool kTcgen05 = false;
};

// Storage of the field B between passes: column blocks of W adjacent columns,
// each block one contiguous [ny][W] array, with the W elements of each of its
// rows permuted by an XOR swizzle. A column pass moves a whole block with one
// bulk copy each way and reads its columns from shared memory without bank
// conflicts; a row pass reads and writes 8W-byte row segments.
//
// P column blocks are in flight per round of a column pass: P = 2 when a
// block of W = 8 columns fills only half of the thread block (512-point
// columns). Each half (slot) then loads, transforms and stores its own column
// block on its own mbarrier, so that all threads work and the copies of one
// half overlap the transforms of the other. (Blocks of 4 columns for
// 1024-point columns, two per round, were measured slower: the column pass
// gained 0.26 us, but the row pass, now reading 32-byte segments from twice
// as many lines, lost 0.5 us.) kPaired = false keeps one block per round (the
// loss kernel's layout).
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

template <int LX, int LY, bool kPaired = true>
struct FieldLayout {
  static constexpr int NX = 1 << LX;
  static constexpr int NY = 1 << LY;
  static constexpr int TY = NY >> 5;          // threads per column transform
  static constexpr int NGY = kThreads / TY;   // column groups per block
  static constexpr int W = cmin(cmin(8, TY), cmin(NGY, NX));
  static constexpr int P = (kPaired && W == 8 && 2 * W * TY == kThreads) ? 2 : 1;  // blocks in flight per round
  static constexpr int LW = ilog2(W);
  static constexpr int S = (W == 1) ? 0 : ilog2(16 / W);
  static constexpr int NBLK = NX / W;
  static constexpr int BLOCK = NY * W;        // elements of one column block
  static_assert(P * BLOCK <= 8192, "the column blocks in flight fit the staging buffer");
  static_assert(P == 1 || W * TY == kThreads / 2, "a slot is half of the block");
  __device__ static constexpr int swz(int y) { return W > 1 ? ((y >> S) & (W - 1)) : 0; }
  // element (row y, column x) of the field
  __device__ static size_t off(int y, int x) {
    return static_cast<size_t>(x >> LW) * BLOCK + y * W + ((x & (W - 1)) ^ swz(y));
  }
  // element (row y, column k) inside one block
  __device__ static int boff(int y, int k) { return y * W + (k ^ swz(y)); }
};

// One pass over rows [lo, hi) (kInit, kRow; LOGN = log2 nx) or column blocks
// [lo, hi) (kCol, kResid, kInitM; LOGN = log2 ny) of mask mb. Returns this
// thread's contribution to the pass's gap sum (FP32: the lines it holds).
template <int LOGN, int LX, int LY, bool HOLD, class TCF>
__device__ __forceinline__ float run_pass(const Params& p, int mb, int kind, bool last, int lo, int hi,
                                           unsigned char* smem, Shared& sh, unsigned& mphase,
                                           const StageTw<LOGN>& tw_rows, const TCF& tcf) {
  // this mask's arrays
  const size_t moff = static_cast<size_t>(mb) * static_cast<size_t>(p.mstride);
  float2* const Bm = p.B + moff;
  const float* const mTm = p.mT + moff;
  using G = GroupT<LOGN>;
  using L = FieldLayout<LX, LY>;
  constexpr int N = G::N;
  constexpr int T = G::T;
  constexpr int LOGT = LOGN - 5;
  constexpr int LOGNG = 8 - LOGT;  // log2(kThreads / T)
  constexpr int NG = 1 << LOGNG;   // groups per block
  static_assert(kThreads == 256, "geometry assumes 256 threads");
  const bool rows = (kind == kInit || kind == kRow);
  const int g = threadIdx.x >> LOGT;
  G grp;
  grp.t = threadIdx.x & (T - 1);
  grp.bar_id = 1 + g;
  grp.sm = reinterpret_cast<float2*>(smem) + g * G::SMEM;
  grp.tw = rows ? p.twx : p.twy;
  const int t = grp.t;
  // stage twiddles: the kernel's register copy for square grids, else
  // loaded once for this pass
  StageTw<LOGN> tw_own;
  if constexpr (!HOLD && !TCF::kEnabled) tw_own.load(grp.tw, t);
  const StageTw<LOGN>& stw = [&]() -> const StageTw<LOGN>& {
    if constexpr (HOLD) return tw_rows;
    else return tw_own;
  }();
  float* ms = reinterpret_cast<float*>(smem + kAmpSmemOffset);
  float2* blk = reinterpret_cast<float2*>(smem + kBlockSmemOffset);
  const int nfft = (kind == kCol || (kind == kRow && !(last && !p.final_resid))) ? 2 : 1;
  const float inv_sqrt_n = p.inv_sqrt_n;
  float acc = 0.f;
  // Tensor-core transforms: this mask's power-of-two operand scales.
  float tc_in = 1.f, tc_out = 32.f;
  if constexpr (TCF::kEnabled) tc_scales(p.nx > p.ny ? p.nx : p.ny, energy_of(p), tc_in, tc_out);
  // One forward transform of the group's vector: on the FP32 ALUs, on the
  // tensor cores through the warp's slice of the exchange buffers (mma.sync),
  // or on the tensor cores of the block's half (tcgen05, all warps at once).
  auto fft = [&](float2(&x)[32]) {
    if constexpr (TCF::kTcgen05) {
      tcf.run(x, tc_in, tc_out);
    } else if constexpr (TCF::kEnabled) {
      tcf.run(x, smem + (threadIdx.x >> 5) * kTcWarpBytes, tc_in, tc_out);
    } else {
      group_fft<LOGN>(x, grp, stw);
    }
  };

  if constexpr (LOGN == LX) {
  if (rows) {
    for (int base = lo; base < hi; base += NG) {
      const int idx = base + g;
      const bool valid = idx < hi;
      const int ridx = valid ? idx : base;  // groups past the end work on a valid copy and store nothing
      float2 v[32];
      if (kind == kInit) {
        // exp(i phi) once per run: a rolled loop through the group's exchange
        // buffer keeps a single copy of sincosf (and atan2f) in the kernel.
        // phi (and p) arrive there first by cp.async, all 32 loads in flight.
        const float* ph = p.phi_in + moff + static_cast<size_t>(ridx) * N + t;
        float2* su = grp.sm + t;
        const float* pp = p.p_slm ? p.p_slm + static_cast<size_t>(ridx) * N + t : nullptr;
        // rolled: the copies do not wait, so all of them are in flight anyway
#pragma unroll 1
        for (int i = 0; i < 32; ++i) cp_async4(&su[T * i].x, ph + T * i);
        if (pp) {
#pragma unroll 1
          for (int i = 0; i < 32; ++i) cp_async4(&su[T * i].y, pp + T * i);
        }
        cp_async_wait_all();
#pragma unroll 1
        for (int i = 0; i < 32; ++i) {
          float s, c;
          const float2 fa = su[T * i];
          sincosf(fa.x, &s, &c);
          const float a = pp ? fa.y : 1.f;  // u0 = p exp(i phi0)
          su[T * i] = make_float2(a * c, a * s);
        }
        if (last && valid) {  // zero iterations: the mask is arg exp(i phi^0)
          float* po = p.phi_out + moff + static_cast<size_t>(idx) * N + t;
#pragma unroll 1
          for (int i = 0; i < 32; ++i) {
            const float2 u = su[T * i];
            const float ph_out = atan2f(u.y, u.x);
            po[T * i] = (ph_out <= -3.14159274f) ? 3.14159274f : ph_out;
          }
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = su[T * i];
        grp.sync();
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = Bm[L::off(ridx, t + T * i)];
        if (kind == kRow && p.p_slm != nullptr) {
          // the laser amplitude of this row, prefetched into the (free in
          // row passes) field staging buffer behind the first transform
          float* sp = reinterpret_cast<float*>(smem + kBlockSmemOffset) + threadIdx.x;
          const float* pp = p.p_slm + static_cast<size_t>(ridx) * N + t;
#pragma unroll 1
          for (int i = 0; i < 32; ++i) cp_async4(sp + kThreads * i, pp + T * i);
        }
      }

      float part = 0.f;
#pragma unroll 1
      for (int h = 0; h < nfft; ++h) {
        fft(v);
        if (h != 0 || kind != kRow) continue;
        // v = swap(IDFT_x(B)) = swap(sqrt(N) P_M u^nu). Gap to S and Eq. (e:PS).
        if (p.p_slm == nullptr) {  // p = 1
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
        } else {
          // SLM amplitude p: u = p v/|v|, gap |P_M u| - p. A rolled loop
          // through the group's exchange buffer keeps this variant out of the
          // unrolled hot code.
          float2* su = grp.sm + t;
          const float* sp = reinterpret_cast<const float*>(smem + kBlockSmemOffset) + threadIdx.x;
#pragma unroll
          for (int i = 0; i < 32; ++i) su[T * i] = v[i];
          cp_async_wait_all();
#pragma unroll 1
          for (int i = 0; i < 32; ++i) {
            const float a = sp[kThreads * i];
            const float2 w = su[T * i];
            const float vx = w.y;
            const float vy = w.x;
            const float a2 = vx * vx + vy * vy;
            const float rs = rsqrtf(a2);
            const float mag = a2 > 0.f ? a2 * rs : 0.f;
            const float d = mag * inv_sqrt_n - a;
            part += d * d;
            const float f = a * rs;
            su[T * i] = a2 > 0.f ? make_float2(vx * f, vy * f) : make_float2(a, 0.f);
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = su[T * i];
          grp.sync();  // the buffer is reused by the next transform's exchange
        }
        if (last) {
          // The mask, once per run: through the group's exchange buffer so
          // that a rolled loop holds the only copy of atan2f.
          float2* su = grp.sm + t;
#pragma unroll
          for (int i = 0; i < 32; ++i) su[T * i] = v[i];
          if (valid) {
            float* po = p.phi_out + moff + static_cast<size_t>(idx) * N + t;
#pragma unroll 1
            for (int i = 0; i < 32; ++i) {
              const float2 u = su[T * i];
              const float ph_out = atan2f(u.y, u.x);
              po[T * i] = (ph_out <= -3.14159274f) ? 3.14159274f : ph_out;
            }
          }
          grp.sync();
        }
      }
      if (valid) acc += part;
      if (valid && (kind == kInit || nfft == 2)) {
#pragma unroll
        for (int i = 0; i < 32; ++i) Bm[L::off(idx, t + T * i)] = v[i];
      }
    }
    return acc;
  }
  }

  // Column passes: P column blocks (W columns, N = ny rows each) per round,
  // one per slot of kThreads / P threads.
  if constexpr (LOGN == LY) {
  constexpr int W = L::W;
  constexpr int P = L::P;
  constexpr int ST = kThreads / P;  // threads of a slot
  constexpr int GS = ST / T;        // groups of a slot
  static_assert(N == L::NY, "column transforms have length ny");
  const int slot = (P == 2) ? static_cast<int>(threadIdx.x >> 7) : 0;
  const int gl = g - slot * GS;                           // group within the slot
  const bool gact = gl < W;                               // this group owns a column
  // some group of this warp owns a column (tcgen05: of this half of the
  // block, whose warps issue their products together)
  const int w_first = (TCF::kTcgen05 ? (((threadIdx.x >> 7) << 7) >> LOGT) : ((threadIdx.x & ~31) >> LOGT)) - slot * GS;
  const bool wact = w_first < W;
  const int gq = gact ? gl : 0;                           // idle groups read a valid column
  const bool leader = (threadIdx.x & (ST - 1)) == 0;      // issues the slot's copies
  uint64_t* const mbar = (P == 2) ? &sh.mbar_s[slot] : &sh.mbar;
  const unsigned pbit = (P == 2) ? (2u << slot) : 1u;     // this mbarrier's phase bit in mphase
  float* const msl = ms + slot * L::BLOCK;                // the slot's amplitude block
  float2* const bsl = blk + slot * L::BLOCK;              // the slot's field block
  // the slot's threads only (the whole block when P == 1)
  auto slot_sync = [&]() {
    if constexpr (P == 2) asm volatile("bar.sync %0, %1;" ::"r"(14 + slot), "n"(ST) : "memory");
    else __syncthreads();
  };
  for (int cb0 = lo; cb0 < hi; cb0 += P) {
    const int cb = cb0 + slot;
    if (cb >= hi) break;  // P = 2: no block left for this slot
    slot_sync();  // the previous round is done with this slot's staging buffers
    const bool from_m = (kind == kInitM);  // transform m itself (the target start)
    const unsigned par = (mphase & pbit) ? 1u : 0u;
    if (leader) {
      bulk_wait_read_all();  // a previous bulk store has read the slot's field block
      fence_proxy_async_smem();
      // the amplitude block is identified by its global address, unique
      // across masks and size classes; the regions of the two layouts of the
      // staging buffer overlap, so loading one invalidates the others
      const float* const msrc = mTm + static_cast<size_t>(cb) * L::BLOCK;
      const float*& resident = (P == 2) ? sh.m_slot[slot] : sh.m_block;
      const bool need_m = (resident != msrc);
      const unsigned bytes_b = from_m ? 0u : L::BLOCK * 8u;
      const unsigned bytes_m = L::BLOCK * 4u;
      mbar_arrive_expect_tx(mbar, bytes_b + (need_m ? bytes_m : 0u));
      if (!from_m) bulk_g2s(bsl, Bm + static_cast<size_t>(cb) * L::BLOCK, bytes_b, mbar);
      // columns cb W .. cb W + W - 1 of m are contiguous in the transposed amplitude
      if (need_m) {
        bulk_g2s(msl, mTm + static_cast<size_t>(cb) * L::BLOCK, bytes_m, mbar);
        if constexpr (P == 2) sh.m_block = nullptr;
        else sh.m_slot[0] = sh.m_slot[1] = nullptr;
      }
      resident = msrc;
      if constexpr (P == 2) {
        sh.pend_s[slot] = 1;
        sh.pend_phase_s[slot] = par;
      } else {
        sh.pending = 1;
        sh.pending_phase = par;
      }
    }
    const bool landed = mbar_wait_bounded(mbar, par);
    mphase ^= pbit;
    if (!landed) {
      fail(p, GS_ETIMEOUT);
    } else if (leader) {
      if constexpr (P == 2) sh.pend_s[slot] = 0;
      else sh.pending = 0;
    }
    if (from_m) {
      // The target start transforms m itself: stage swap((m, 0)) in the field
      // layout, so the forward DFT below yields swap(IDFT_y(m)).
      for (int e = threadIdx.x & (ST - 1); e < L::BLOCK; e += ST) {
        const int k = e % W;
        const int y = e / W;
        bsl[L::boff(y, k)] = make_float2(0.f, msl[k * N + y]);
      }
      slot_sync();
    }
    if (wact) {
      float2 v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = bsl[L::boff(t + T * i, gq)];
      float part = 0.f;
#pragma unroll 1
      for (int h = 0; h < nfft; ++h) {
        fft(v);
        if (h != 0 || from_m) continue;
        // v = Y = F u^nu along this column. Residual and Eq. (e:Mhat).
        const float* mcol = msl + gq * N + t;
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
      }
      if (gact) acc += part;
      if ((kind == kCol || from_m) && gact) {
#pragma unroll
        for (int i = 0; i < 32; ++i) bsl[L::boff(t + T * i, gl)] = v[i];
      }
    }
    if (kind == kCol || from_m) {
      slot_sync();
      if (leader) {
        fence_proxy_async_smem();
        bulk_s2g(Bm + static_cast<size_t>(cb) * L::BLOCK, bsl, L::BLOCK * 8u);
        bulk_commit();
      }
    }
  }
  // the field must be in global memory before the grid barrier releases the next pass
  if ((kind == kCol || kind == kInitM) && leader) bulk_wait_all();
  }
  return acc;
}

// Before leaving after a failure, give a bulk copy that may still target this
// block's shared memory a bounded time to land.
static __device__ void drain_copies(Shared& sh) {
  if (threadIdx.x == 0 && sh.pending) mbar_wait_bounded(&sh.mbar, sh.pending_phase);
  for (int s = 0; s < 2; ++s)
    if (threadIdx.x == 128u * s && sh.pend_s[s]) mbar_wait_bounded(&sh.mbar_s[s], sh.pend_phase_s[s]);
  __syncthreads();
}

// m = s sqrt(I) for this block's columns, written transposed ([nx][ny]) so
// that the column pass reads it contiguously.
static __device__ void build_amplitude(const Params& p, int mb, float s, unsigned char* smem) {
  const size_t moff = static_cast<size_t>(mb) * static_cast<size_t>(p.mstride);
  const float* const Im = p.I + moff;
  float* const mTm = p.mT + moff;
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
      if (k < wcur) blk[y * (W + 1) + k] = Im[static_cast<size_t>(y) * p.nx + base + k];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < wcur * p.ny; e += kThreads) {
      const int k = e >> p.logny;
      const int y = e & (p.ny - 1);
      mTm[static_cast<size_t>(base + k) * p.ny + y] = s * sqrtf(blk[y * (W + 1) + k]);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The kernels. A launch iterates one or more *size classes*: each class is a
// Params (a batch of masks of one grid, with its own arrays and partial-sum
// region); all classes share the barrier, status and abort words and pass
// through the same schedule, one grid barrier per pass. Shared state of mask
// mb of a class lives at index base + mb of the block's Shared arrays.

// A0, part 1: this block's FP64 share of sum I for every mask of the class.
// A non-finite or negative pixel poisons the sum with NaN.
static __device__ __forceinline__ void a0_partials(const Params& p, Shared& sh) {
  const int G = gridDim.x;
  const int b = blockIdx.x;
  const int r0 = split(b, G, p.ny);
  const int r1 = split(b + 1, G, p.ny);
  const int cnt = (r1 - r0) * p.nx;
  for (int mb = 0; mb < p.batch; ++mb) {
    const float* I = p.I + static_cast<size_t>(mb) * static_cast<size_t>(p.mstride) + static_cast<size_t>(r0) * p.nx;
    double acc = 0.0;
    bool bad = false;
    for (int e = threadIdx.x; e < cnt; e += kThreads) {
      const float x = I[e];
      bad |= !(x >= 0.f && x <= FLT_MAX);
      acc += static_cast<double>(x);
    }
    if (__syncthreads_or(bad)) acc = __longlong_as_double(0x7ff8000000000000ll);
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) p.partials[static_cast<size_t>(mb) * G + b] = tot;
  }
}

// A0, part 2 (after a grid barrier): validity and scale sqrt(sum p^2 / sum I)
// of every mask, the same in every block (each reduces the same partials in
// the same order). Rejected masks get NaN gaps and GS_ENUMERIC; they are
// skipped from then on. (The tensor-core forms keep their FP16 operands in
// range with a power-of-two scale per mask, tc_scales, so no energy is too
// large for them.) Returns the number of rejected masks.
static __device__ __forceinline__ int a0_scales(const Params& p, Shared& sh, int base) {
  const int b = blockIdx.x;
  if (threadIdx.x < 32) {
    for (int mb = 0; mb < p.batch; ++mb) {
      const double total = warp_slot_sum(p, mb);
      if (threadIdx.x == 0) {
        const double ep = energy_of(p);
        const bool bad = !(total > 0.0) || !(total <= DBL_MAX) || !(ep > 0.0) || !(ep <= DBL_MAX);
        sh.bad[base + mb] = bad ? 1 : 0;
        if (b == 0) p.mask_flags[mb] = bad ? 1 : 0;  // for later launches of the run
        sh.scale[base + mb] = bad ? 0.f : static_cast<float>(sqrt(ep / total));
      }
    }
  }
  __syncthreads();
  int nbad = 0;
  for (int mb = 0; mb < p.batch; ++mb) nbad += sh.bad[base + mb];
  if (nbad > 0 && b == 0) {
    // Masks with an invalid target are skipped: phase untouched, gaps NaN.
    if (threadIdx.x == 0) fail_status(p, GS_ENUMERIC);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const int nr = p.iters + (p.final_resid ? 1 : 0);
    for (int mb = 0; mb < p.batch; ++mb) {
      if (!sh.bad[base + mb]) continue;
      if (p.r_out)
        for (int e = threadIdx.x; e < nr; e += kThreads) p.r_out[static_cast<size_t>(mb) * p.rstride + e] = nan;
      if (p.g_out)
        for (int e = threadIdx.x; e < p.iters; e += kThreads) p.g_out[static_cast<size_t>(mb) * p.gstride + e] = nan;
    }
  }
  return nbad;
}

// Later launches of a run: the invalid masks were flagged by the first.
static __device__ __forceinline__ void restore_flags(const Params& p, Shared& sh, int base) {
  if (threadIdx.x == 0)
    for (int mb = 0; mb < p.batch; ++mb) sh.bad[base + mb] = p.mask_flags[mb];
}

template <int LX, int LY = LX>
__device__ __forceinline__ void build_amplitudes(const Params& p, Shared& sh, int base, unsigned char* smem) {
  for (int mb = 0; mb < p.batch; ++mb)
    if (!sh.bad[base + mb]) {
      if constexpr (LX == 0) gen_build_amplitude(p, mb, sh.scale[base + mb]);
      else if constexpr (is_rg_side(LX)) rg_build_amplitude<LX, LY>(p, mb, sh.scale[base + mb], smem);
      else build_amplitude(p, mb, sh.scale[base + mb], smem);
    }
}

// Pass q0 of the schedule [init] (col, row) x nit [resid]: its kind, whether
// it ends the run, and the partial-sum slot of its gap (-1: none). Pass q
// after the init passes sums into slot 1 + q.
struct PassInfo {
  int kind;
  int slot;
  bool last;
};

static __device__ __forceinline__ int pass_count(const Params& p) {
  const int nit = p.it1 - p.it0;
  const int resid = (p.do_final && p.final_resid) ? 1 : 0;
  const int ninit = p.do_init ? (p.init_target ? 2 : 1) : 0;  // target start: columns then rows
  return ninit + 2 * nit + resid;
}

static __device__ __forceinline__ PassInfo pass_info(const Params& p, int q0) {
  const int nit = p.it1 - p.it0;
  const int ninit = p.do_init ? (p.init_target ? 2 : 1) : 0;
  const int q = q0 - ninit;
  PassInfo f{kCol, -1, false};
  if (q < 0) {
    f.kind = !p.init_target ? kInit : (q == -2 ? kInitM : kRow);
    f.last = p.do_final && p.iters == 0 && q == -1;
  } else if (q < 2 * nit) {
    f.kind = (q & 1) ? kRow : kCol;
    f.slot = 1 + q;
    f.last = (f.kind == kRow) && p.do_final && (p.it0 + (q >> 1) == p.iters - 1);
  } else {
    f.kind = kResid;
    f.slot = 1 + q;
  }
  return f;
}

// One pass over the valid masks [w0, w1) of a class. The work units of those
// masks (rows, or column blocks) form one sequence split evenly over the
// blocks, so that small masks of a batch do not leave blocks idle; a block
// works through its share mask by mask and writes the FP64 partial of each
// mask's gap to its slot (zero for the masks it does not touch).
template <int LX, int LY, bool HOLD, class TCF, class TW>
__device__ __forceinline__ void class_pass(const Params& p, Shared& sh, int base, int w0, int w1, const PassInfo& f,
                                           unsigned char* smem, unsigned& mphase, const TW& tw_rows,
                                           const TCF& tcf) {
  const bool rows = (f.kind == kInit || f.kind == kRow);
  int per;  // units of one mask
  if constexpr (LX == 0) per = rows ? p.ny : (p.nx + kGenTeams - 1) / kGenTeams;
  else if constexpr (is_rg_side(LX)) per = rows ? p.ny : LX / RgLayout<LX, LY>::W;
  else per = rows ? p.ny : FieldLayout<LX, LY>::NBLK;
  const int G = gridDim.x;
  int lo, hi, m0, m1;
  if (w1 - w0 == 1) {  // one mask: its own share, no mask boundaries
    lo = split(blockIdx.x, G, per);
    hi = split(blockIdx.x + 1, G, per);
    m0 = w0;
    m1 = w1;
  } else {
    const int total = per * (w1 - w0);
    lo = split(blockIdx.x, G, total);
    hi = split(blockIdx.x + 1, G, total);
    m0 = w0 + lo / per;
    m1 = w0 + (hi + per - 1) / per;  // masks [m0, m1) meet [lo, hi)
    if (f.slot >= 0 && threadIdx.x == 0)
      for (int mb = w0; mb < w1; ++mb)
        if (mb < m0 || mb >= m1) p.partials[(static_cast<size_t>(f.slot) * p.batch + mb) * G + blockIdx.x] = 0.0;
  }
  for (int mb = m0; mb < m1; ++mb) {
    if (sh.bad[base + mb]) continue;
    const int slo = max(lo, (mb - w0) * per) - (mb - w0) * per;
    const int shi = min(hi, (mb - w0 + 1) * per) - (mb - w0) * per;
    float a;
    if constexpr (LX == 0) {
      a = run_pass_gen(p, mb, f.kind, f.last, slo, shi, smem);
    } else if constexpr (is_rg_side(LX)) {
      a = run_pass_rg<LX, LY>(p, mb, f.kind, f.last, slo, shi, smem, sh, mphase);
    } else if constexpr (LX == LY) {
      a = run_pass<LX, LX, LY, HOLD>(p, mb, f.kind, f.last, slo, shi, smem, sh, mphase, tw_rows, tcf);
    } else {
      const StageTw<LY> none{};
      a = rows ? run_pass<LX, LX, LY, false>(p, mb, f.kind, f.last, slo, shi, smem, sh, mphase, tw_rows, tcf)
               : run_pass<LY, LX, LY, false>(p, mb, f.kind, f.last, slo, shi, smem, sh, mphase, none, tcf);
    }
    if (f.slot >= 0) {
      const double tot = block_sum_f(a, sh);
      if (threadIdx.x == 0) p.partials[(static_cast<size_t>(f.slot) * p.batch + mb) * G + blockIdx.x] = tot;
    }
  }
}

// Gaps: r from column passes, g from row passes, in FP64, for every valid
// mask of a class (block b reduces slots b, b + G, ...).
static __device__ __forceinline__ void final_gaps(const Params& p, Shared& sh, int base) {
  const int G = gridDim.x;
  const int nit = p.it1 - p.it0;
  const int resid = (p.do_final && p.final_resid) ? 1 : 0;
  const int nslots = 2 * nit + resid;
  if (threadIdx.x < 32) {
    for (int s = blockIdx.x; s < nslots * p.batch; s += G) {
      const int slot = 1 + s / p.batch;
      const int mb = s % p.batch;
      if (sh.bad[base + mb]) continue;
      const double sum = warp_slot_sum(p, slot * p.batch + mb);
      if (threadIdx.x == 0) {
        const double val = sqrt(sum / energy_of(p));
        const int q = slot - 1;
        if (q < 2 * nit) {
          const int nu = p.it0 + (q >> 1);
          if ((q & 1) == 0) {
            if (p.r_out) p.r_out[static_cast<size_t>(mb) * p.rstride + nu] = val;
          } else {
            if (p.g_out) p.g_out[static_cast<size_t>(mb) * p.gstride + nu] = val;
          }
        } else if (p.r_out) {
          p.r_out[static_cast<size_t>(mb) * p.rstride + p.iters] = val;
        }
      }
    }
  }
}

static __device__ __forceinline__ void block_setup(Shared& sh) {
  if (threadIdx.x == 0) {
    mbar_init(&sh.mbar, 1);
    mbar_init(&sh.mbar_s[0], 1);
    mbar_init(&sh.mbar_s[1], 1);
    fence_barrier_init();
    sh.pending = 0;
    sh.m_block = nullptr;
    sh.m_slot[0] = sh.m_slot[1] = nullptr;
    sh.pend_s[0] = sh.pend_s[1] = 0;
  }
  __syncthreads();
}

// The schedule of one size class (every grid): A0, then the passes, then the
// gaps. Returns early (in every thread of the block) when a grid barrier gave
// up or every mask was rejected.
template <int LX, int LY, bool kHold, class TCF, class TW>
__device__ __forceinline__ void iterate_class(const Params& p, Shared& sh, unsigned char* smem,
                                              const TW& tw_rows, const TCF& tcf) {
  unsigned target = 0;
  unsigned mphase = 0;
  block_setup(sh);
  if constexpr (LX == 0) gen_load_twiddles(p, smem);  // sides that are not powers of two
  if constexpr (is_rg_side(LX)) rg_load_twiddles<LX, LY>(p, smem);

  if (p.do_init) {
    a0_partials(p, sh);
    if (!grid_sync(p, target, sh)) return;
    const int nbad = a0_scales(p, sh, 0);
    if (nbad == p.batch) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(p.abort_flag, 1);  // later launches of the run
      return;
    }
    build_amplitudes<LX, LY>(p, sh, 0, smem);
    // the target start transforms m in its first pass, reading columns that
    // other blocks built
    if (p.init_target && !grid_sync(p, target, sh)) return;
  } else {
    restore_flags(p, sh, 0);
  }
  __syncthreads();

  const int npass = pass_count(p);
  const int gsz = p.group > 0 ? p.group : p.batch;
  unsigned long long* const tr = (p.trace != nullptr && threadIdx.x == 0) ? p.trace + 2 * blockIdx.x : nullptr;
  if (tr) tr[0] = tr[1] = global_ns();
  for (int w0 = 0; w0 < p.batch; w0 += gsz) {  // mask groups, each through the whole schedule
    const int w1 = min(p.batch, w0 + gsz);
    for (int q0 = 0; q0 < npass; ++q0) {
      class_pass<LX, LY, kHold>(p, sh, 0, w0, w1, pass_info(p, q0), smem, mphase, tw_rows, tcf);
      // pass timestamps: work done, then released by the barrier
      unsigned long long* const trq = tr ? tr + static_cast<size_t>(2 * (1 + q0)) * gridDim.x : nullptr;
      if (trq) trq[0] = global_ns();
      if (!grid_sync(p, target, sh)) {
        drain_copies(sh);
        return;
      }
      if (trq) trq[1] = global_ns();
    }
  }
  final_gaps(p, sh, 0);
}

// One size class per launch (every grid).
template <int LX, int LY, bool TC = false>
__global__ void __launch_bounds__(kThreads, 1) gs_iterate(const Params p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shared sh;
  if (*reinterpret_cast<volatile int*>(p.abort_flag) != 0) return;  // an earlier chunk failed
  constexpr bool kHold = LX > 0 && LX == LY && !TC;
  StageTw<LX> tw_rows;  // square grids: stage twiddles held for the whole run
  if constexpr (kHold) tw_rows.load(p.twx, threadIdx.x & ((1 << (LX - 5)) - 1));
  // Tensor-core transforms: the block's tables, then the DFT-matrix fragments
  // held in registers for the whole run.
  static_assert(!TC || LX == LY, "tensor-core kernels are square");
  constexpr int kR = TC ? (1 << (LX > 5 ? LX - 5 : 0)) : 32;
  TcStage1 s1;
  TcStage2<kR> s2;
  const float2* tctw = reinterpret_cast<const float2*>(smem + kTcTwOffset);
  if constexpr (TC) {
    tc_build_tables<LX>(reinterpret_cast<float2*>(smem + kTcTwOffset), reinterpret_cast<float2*>(smem + kTcCsOffset));
    __syncthreads();
    s1.load(reinterpret_cast<const float2*>(smem + kTcCsOffset));
    s2.load(reinterpret_cast<const float2*>(smem + kTcCsOffset));
  }
  const auto tcf = [&]() {
    if constexpr (TC) return TcFft<LX>{s1, s2, tctw};
    else return NoTc{};
  }();
  iterate_class<LX, LY, kHold>(p, sh, smem, tw_rows, tcf);
}

// The tensor-core form on tcgen05 (square 256, 512, 1024): the same schedule
// with every transform issued by the block's halves as products on the
// tensor cores (gs_tc5.cuh). Warp 0 holds the block's TMEM columns from the
// start of the launch to its end, on every exit path.
constexpr int kTc5Offset = kBlockSmemOffset + kBlockSmemBytes;  // after the amplitude and field blocks

template <int L, bool BF16>
__global__ void __launch_bounds__(kThreads, 1) gs_iterate_tc5(const Params p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shared sh;
  __shared__ uint64_t tc_mbar[2];
  __shared__ unsigned tc_tmem;
  if (*reinterpret_cast<volatile int*>(p.abort_flag) != 0) return;  // an earlier chunk failed
  static_assert(2 * kTc5HalfStride == kGroupSmemBytes, "the A operands fill the exchange area");
  unsigned char* abuf = smem;  // the exchange area (gs_tc5.cuh)
  unsigned char* tabs = smem + kTc5Offset;
  tc5_build_tables<L, BF16>(tabs, tabs + kTc5B2Offset, reinterpret_cast<float2*>(tabs + kTc5TwOffset));
  if (threadIdx.x == 0) {
    mbar_init(&tc_mbar[0], 1);
    mbar_init(&tc_mbar[1], 1);
    fence_barrier_init();
  }
  if ((threadIdx.x >> 5) == 0) tc5_alloc(&tc_tmem);
  fence_proxy_async_smem();  // the DFT matrices are read by the tensor cores
  tc5_fence_before();
  __syncthreads();
  tc5_fence_after();
  unsigned phase = 0;
  const Tc5Fft<L, BF16> tcf{abuf, smem_u32(tabs), smem_u32(tabs + kTc5B2Offset),
                            reinterpret_cast<const float2*>(tabs + kTc5TwOffset), tc_mbar, tc_tmem, &phase, &p};
  const StageTw<L> none{};
  iterate_class<L, L, false>(p, sh, smem, none, tcf);
  tc5_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tc5_dealloc(tc_tmem);
}

template <int C, bool TC>
__device__ __forceinline__ void mixed_class_pass(const MixedParams& mp, Shared& sh, int w0, int w1, const PassInfo& f,
                                                 unsigned char* smem, unsigned& mphase, const TcStage1& s1,
                                                 const TcStage2<8 << C>& s2) {
  constexpr int L = 8 + C;
  const Params& p = mp.cls[C];
  const int base = (C > 0 ? mp.cls[0].batch : 0) + (C > 1 ? mp.cls[1].batch : 0);
  const StageTw<L> none{};
  if constexpr (TC) {
    const TcFft<L> tcf{s1, s2, reinterpret_cast<const float2*>(smem + kTcTwOffset + C * kTcTwBytes)};
    class_pass<L, L, false>(p, sh, base, w0, w1, f, smem, mphase, none, tcf);
  } else {
    class_pass<L, L, false>(p, sh, base, w0, w1, f, smem, mphase, none, NoTc{});
  }
}

// The schedule of a mixed launch (the tcgen05 form; gs_iterate_mixed writes
// the same out): A0 for every class, then the classes one after the other,
// each (in mask groups) through the whole schedule of passes;
// `pass(c, w0, w1, f, mphase)` runs one pass of class c. Returns early when a
// barrier gave up or every mask was rejected.
template <class PassFn>
__device__ __forceinline__ void iterate_mixed(const MixedParams& mp, Shared& sh, unsigned char* smem, PassFn&& pass) {
  const Params& p0 = mp.cls[0];  // barrier, status, abort flag, schedule
  unsigned target = 0;
  unsigned mphase = 0;
  block_setup(sh);
  const int total = mp.cls[0].batch + mp.cls[1].batch + mp.cls[2].batch;
  const int base1 = mp.cls[0].batch, base2 = base1 + mp.cls[1].batch;

  if (p0.do_init) {
    for (int c = 0; c < 3; ++c) a0_partials(mp.cls[c], sh);
    if (!grid_sync(p0, target, sh)) return;
    const int nbad = a0_scales(mp.cls[0], sh, 0) + a0_scales(mp.cls[1], sh, base1) + a0_scales(mp.cls[2], sh, base2);
    if (nbad == total) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(p0.abort_flag, 1);
      return;
    }
    build_amplitudes<8>(mp.cls[0], sh, 0, smem);
    build_amplitudes<9>(mp.cls[1], sh, base1, smem);
    build_amplitudes<10>(mp.cls[2], sh, base2, smem);
    // the target start transforms m in its first pass, reading columns that
    // other blocks built
    if (p0.init_target && !grid_sync(p0, target, sh)) return;
  } else {
    restore_flags(mp.cls[0], sh, 0);
    restore_flags(mp.cls[1], sh, base1);
    restore_flags(mp.cls[2], sh, base2);
  }
  __syncthreads();

  // Mask groups (each class's group size keeps a group's fields in L2), each
  // through the whole schedule; classes one after the other.
  const int npass = pass_count(p0);
  for (int c = 0; c < 3; ++c) {
    const Params& pc = mp.cls[c];
    const int gsz = pc.group > 0 ? pc.group : pc.batch;
    for (int w0 = 0; w0 < pc.batch; w0 += gsz) {
      const int w1 = min(pc.batch, w0 + gsz);
      for (int q0 = 0; q0 < npass; ++q0) {
        pass(c, w0, w1, pass_info(p0, q0), mphase);
        if (!grid_sync(p0, target, sh)) {
          drain_copies(sh);
          return;
        }
      }
    }
  }
  final_gaps(mp.cls[0], sh, 0);
  final_gaps(mp.cls[1], sh, base1);
  final_gaps(mp.cls[2], sh, base2);
}

template <bool TC>
__global__ void __launch_bounds__(kThreads, 1) gs_iterate_mixed(const MixedParams mp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shared sh;
  if (*reinterpret_cast<volatile int*>(mp.cls[0].abort_flag) != 0) return;
  TcStage1 s1;
  TcStage2<8> s2a;
  TcStage2<16> s2b;
  TcStage2<32> s2c;
  if constexpr (TC) {
    float2* cs = reinterpret_cast<float2*>(smem + kTcTwOffset + 3 * kTcTwBytes);
    tc_build_tables<8>(reinterpret_cast<float2*>(smem + kTcTwOffset), cs);
    tc_build_tables<9>(reinterpret_cast<float2*>(smem + kTcTwOffset + kTcTwBytes), cs);
    tc_build_tables<10>(reinterpret_cast<float2*>(smem + kTcTwOffset + 2 * kTcTwBytes), cs);
    __syncthreads();
    s1.load(cs);
    s2a.load(cs);
    s2b.load(cs);
  }
  // The schedule of iterate_mixed, written out: passing the register-held
  // DFT fragments through a closure moved them to local memory.
  const Params& p0 = mp.cls[0];
  unsigned target = 0;
  unsigned mphase = 0;
  block_setup(sh);
  const int total = mp.cls[0].batch + mp.cls[1].batch + mp.cls[2].batch;
  const int base1 = mp.cls[0].batch, base2 = base1 + mp.cls[1].batch;
  if (p0.do_init) {
    for (int c = 0; c < 3; ++c) a0_partials(mp.cls[c], sh);
    if (!grid_sync(p0, target, sh)) return;
    const int nbad = a0_scales(mp.cls[0], sh, 0) + a0_scales(mp.cls[1], sh, base1) + a0_scales(mp.cls[2], sh, base2);
    if (nbad == total) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(p0.abort_flag, 1);
      return;
    }
    build_amplitudes<8>(mp.cls[0], sh, 0, smem);
    build_amplitudes<9>(mp.cls[1], sh, base1, smem);
    build_amplitudes<10>(mp.cls[2], sh, base2, smem);
    // the target start transforms m in its first pass, reading columns that
    // other blocks built
    if (p0.init_target && !grid_sync(p0, target, sh)) return;
  } else {
    restore_flags(mp.cls[0], sh, 0);
    restore_flags(mp.cls[1], sh, base1);
    restore_flags(mp.cls[2], sh, base2);
  }
  __syncthreads();
  const int npass = pass_count(p0);
  for (int c = 0; c < 3; ++c) {
    const Params& pc = mp.cls[c];
    const int gsz = pc.group > 0 ? pc.group : pc.batch;
    for (int w0 = 0; w0 < pc.batch; w0 += gsz) {
      const int w1 = min(pc.batch, w0 + gsz);
      for (int q0 = 0; q0 < npass; ++q0) {
        const PassInfo f = pass_info(p0, q0);
        if (c == 0) mixed_class_pass<0, TC>(mp, sh, w0, w1, f, smem, mphase, s1, s2a);
        else if (c == 1) mixed_class_pass<1, TC>(mp, sh, w0, w1, f, smem, mphase, s1, s2b);
        else mixed_class_pass<2, TC>(mp, sh, w0, w1, f, smem, mphase, s1, s2c);
        if (!grid_sync(p0, target, sh)) {
          drain_copies(sh);
          return;
        }
      }
    }
  }
  final_gaps(mp.cls[0], sh, 0);
  final_gaps(mp.cls[1], sh, base1);
  final_gaps(mp.cls[2], sh, base2);
}

// The mixed launch with tcgen05 transforms: one TMEM allocation for the
// launch, the 32-point matrix shared by the three lengths, an R-point matrix
// and a twiddle table per length (kMixedTc5SmemBytes after the kernel's own
// shared memory).
// offset of the R-point matrix of class c (R = 8 << c) in the tables
__host__ __device__ constexpr int mixed_b2_offset(int c) {
  return 2 * tc5_form_bytes(32) + (c > 0 ? 2 * tc5_form_bytes(8) : 0) + (c > 1 ? 2 * tc5_form_bytes(16) : 0);
}
constexpr int kMixedTwOffset = 4 * tc5_form_bytes(32) + 2 * tc5_form_bytes(8) + 2 * tc5_form_bytes(16);
static_assert(kMixedTwOffset + 3 * kTc5TwBytes == kMixedTc5ExtraSmemBytes, "mixed tcgen05 tables match the launch size");

template <int C, bool BF16>
__device__ __forceinline__ void mixed_class_pass_tc5(const MixedParams& mp, Shared& sh, int w0, int w1,
                                                     const PassInfo& f, unsigned char* smem, unsigned& mphase,
                                                     const Tc5Fft<8 + C, BF16>& tcf) {
  constexpr int L = 8 + C;
  const int base = (C > 0 ? mp.cls[0].batch : 0) + (C > 1 ? mp.cls[1].batch : 0);
  const StageTw<L> none{};
  class_pass<L, L, false>(mp.cls[C], sh, base, w0, w1, f, smem, mphase, none, tcf);
}

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) gs_iterate_mixed_tc5(const MixedParams mp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shared sh;
  __shared__ uint64_t tc_mbar[2];
  __shared__ unsigned tc_tmem;
  const Params& p0 = mp.cls[0];
  if (*reinterpret_cast<volatile int*>(p0.abort_flag) != 0) return;
  static_assert(2 * kTc5HalfStride == kGroupSmemBytes, "the A operands fill the exchange area");
  unsigned char* tabs = smem + kTc5Offset;
  float2* tw = reinterpret_cast<float2*>(tabs + kMixedTwOffset);
  tc5_build_tables<8, BF16>(tabs, tabs + mixed_b2_offset(0), tw);
  tc5_build_tables<9, BF16>(nullptr, tabs + mixed_b2_offset(1), tw + 1024);
  tc5_build_tables<10, BF16>(nullptr, tabs + mixed_b2_offset(2), tw + 2048);
  if (threadIdx.x == 0) {
    mbar_init(&tc_mbar[0], 1);
    mbar_init(&tc_mbar[1], 1);
    fence_barrier_init();
  }
  if ((threadIdx.x >> 5) == 0) tc5_alloc(&tc_tmem);
  fence_proxy_async_smem();  // the DFT matrices are read by the tensor cores
  tc5_fence_before();
  __syncthreads();
  tc5_fence_after();
  unsigned phase = 0;  // one parity per half, shared by the three lengths (their products run in turn)
  const unsigned b1 = smem_u32(tabs);
  const Tc5Fft<8, BF16> t8{smem, b1, smem_u32(tabs + mixed_b2_offset(0)), tw, tc_mbar, tc_tmem, &phase, &p0};
  const Tc5Fft<9, BF16> t9{smem, b1, smem_u32(tabs + mixed_b2_offset(1)), tw + 1024, tc_mbar, tc_tmem, &phase, &p0};
  const Tc5Fft<10, BF16> t10{smem, b1, smem_u32(tabs + mixed_b2_offset(2)), tw + 2048, tc_mbar, tc_tmem, &phase, &p0};
  iterate_mixed(mp, sh, smem, [&](int c, int w0, int w1, const PassInfo& f, unsigned& mphase) {
    if (c == 0) mixed_class_pass_tc5<0, BF16>(mp, sh, w0, w1, f, smem, mphase, t8);
    else if (c == 1) mixed_class_pass_tc5<1, BF16>(mp, sh, w0, w1, f, smem, mphase, t9);
    else mixed_class_pass_tc5<2, BF16>(mp, sh, w0, w1, f, smem, mphase, t10);
  });
  tc5_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tc5_dealloc(tc_tmem);
}

}  // namespace gsk
