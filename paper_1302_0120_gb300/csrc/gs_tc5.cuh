// gs_tc5.cuh -- the 1024-point DFT of the tensor-core form on the fifth-
// generation tensor cores (tcgen05): FP16 or BF16 operands in shared memory,
// FP32 accumulators in tensor memory (TMEM).
//
// Same arithmetic as gs_tc.cuh (the four-step factorisation 1024 = 32 x 32,
// both stages dense products with the real form of the 32-point DFT matrix),
// but batched: the four warps of one half of the block hold four lines (one
// line per warp, lane t holding x[t + 32 i], i = 0..31, the thread layout of
// the FP32 transforms), and each stage is ONE product of the half's 128 rows
// (line, t) with the 64 x 64 real-form matrix, issued by one thread as four
// tcgen05.mma (M = 128, N = 64, K = 16) into 64 TMEM columns:
//
//   stage 1  D1[(w, t)][k1]   = sum_i  x_w[t + 32 i] W_32^{i k1}        (A K-major: row (w, t) = [re x_i | im x_i])
//   twiddle  Z[(w, k1)][t]    = D1[(w, t)][k1] W_1024^{k1 t} / 32       (epilogue of tcgen05.ld, FP32)
//   stage 2  D2[(w, k1)][k2]  = sum_t  Z[(w, k1)][t] W_32^{t k2}         (A MN-major: column t = [re | im])
//            X_w[k1 + 32 k2]  = 32 D2[(w, k1)][k2]
//
// Lane t of warp w reads TMEM lane 32 (w mod 4) + t, i.e. row (w, t) of D1 and
// row (w, k1 = t) of D2, so the result X_w[t + 32 k2] lands in the thread
// layout the transform started from. The two halves of the block run their
// products independently (own mbarrier, own TMEM columns, own named
// barrier), so one half's tensor-core latency overlaps the other's FP32
// epilogue.
//
// Shared-memory operands use the canonical no-swizzle layout: 8 x 16-byte
// core matrices, 128 bytes each. K-major: core (m/8, k/8) at ((m/8) 8 +
// k/8) 128, row m mod 8 at 16 (m mod 8); the leading byte offset (next core
// along K) is 128, the stride byte offset (next core along M or N) 1024.
// MN-major: core (m/8, k/8) at ((k/8) 16 + m/8) 128, row k mod 8 at
// 16 (k mod 8), m mod 8 at 2 (m mod 8); leading byte offset (along K) 2048,
// stride byte offset (along M) 128.
//
// Range: the caller passes a power-of-two input scale that keeps every FP16
// operand below 2^15 (stage-1 inputs are bounded by sqrt(n sum p^2), stage-1
// outputs by 32 times that, hence the 1/32 in the twiddles) and the inverse
// scale times 32 for the output; BF16 has FP32's range and uses the same
// scales. Every wait on an mbarrier is bounded (1 s), after which the run is
// failed with GS_ETIMEOUT.
//
// BF16 keeps 8 significant bits (unit roundoff 2^-8 against FP16's 2^-11): one
// BF16 product per stage leaves about 8e-3 relative error per GS step. The
// BF16 form therefore splits every operand into a rounded part and the
// rounded remainder, x = hi + lo (both BF16, |lo| <= 2^-8 |x|), and forms
// hi_A hi_B + hi_A lo_B + lo_A hi_B (the dropped lo_A lo_B is below 2^-16
// relative): three products per K step, about 16 significant bits.
//
// Shared memory: the A operands of half h occupy bytes [h 33792, h 33792 +
// 32768) of the block's FFT exchange area (A_hi, then A_lo), the region
// that warps 4h..4h+3 use as scratch outside the transform; each transform
// therefore starts with a barrier of its half.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "gs_common.cuh"
#include "gs_fft.cuh"
#include "gs_tma.cuh"

namespace gsk {

// Shared memory of the tcgen05 transform after the iteration kernel's own:
// the real-form DFT matrix (hi, then lo: 8 KiB each) and the 8 KiB twiddle
// table [k1][t]. The A operands live in the exchange area (kTc5HalfStride
// bytes per half: A_hi 16 KiB, A_lo 16 KiB).
constexpr int kTc5HalfStride = 4 * 32 * 33 * 8;  // the exchange buffers of four warps
constexpr int kTc5AloOffset = 16384;
constexpr int kTc5BBytes = 64 * 64 * 2;
constexpr int kTc5TwBytes = 32 * 32 * 8;
constexpr int kTc5SmemBytes = 2 * kTc5BBytes + kTc5TwBytes;
static_assert(kTc5SmemBytes == kTc5ExtraSmemBytes, "tcgen05 tables match the launch size");
static_assert(2 * kTc5AloOffset <= kTc5HalfStride, "both A operands of a half fit its exchange buffers");
constexpr int kTc5TmemCols = 128;  // two halves x 64 FP32 columns

__device__ __forceinline__ uint64_t tc5_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (static_cast<uint64_t>(1) << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, FP16 (0) or BF16 (1)
// operands, A K-major (0) or MN-major (1), B K-major, N = 64, M = 128.
__host__ __device__ constexpr unsigned tc5_idesc(bool bf16, bool a_mn) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((a_mn ? 1u : 0u) << 15) |
         ((64u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tc5_mma(unsigned d_tmem, uint64_t adesc, uint64_t bdesc, unsigned idesc,
                                        unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc5_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc5_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc5_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 FP32 columns of this warp's 32 TMEM lanes starting at taddr.
__device__ __forceinline__ void tc5_ld16(float (&d)[16], unsigned taddr) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) d[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tc5_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Warp 0 allocates the TMEM columns of the block (the address lands in *slot).
__device__ __forceinline__ void tc5_alloc(unsigned* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "n"(kTc5TmemCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc5_dealloc(unsigned tmem) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTc5TmemCols) : "memory");
}

template <bool BF16>
__device__ __forceinline__ uint32_t tc5_pack(float lo, float hi) {
  uint32_t u;
  if constexpr (BF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    memcpy(&u, &h, 4);
  } else {
    const __half2 h = __floats2half2_rn(lo, hi);
    memcpy(&u, &h, 4);
  }
  return u;
}

// The block's constant tables: the real form of the 32-point DFT matrix as
// the K-major B operand (row n, column K): n < 32 gives Re y_n, n >= 32 gives
// Im y_{n-32}; K < 32 multiplies re x_K, K >= 32 im x_{K-32}:
//   B[n][K] = cos, B[n][32+K] = sin, B[32+n][K] = -sin, B[32+n][32+K] = cos
// of 2 pi n K / 32 (since W (a + i b) = (c a + s b) + i (c b - s a) for
// W = c - i s); and the stage twiddles tw[k1][t] = W_1024^{k1 t} / 32.
template <bool BF16>
__device__ void tc5_build_tables(unsigned char* bmat, float2* tw) {
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int n = e >> 6, K = e & 63;
    const int kk = K & 31, nn = n & 31;
    float s, c;
    sincospif(static_cast<float>((nn * kk) & 31) / 16.0f, &s, &c);
    const float val = ((n < 32) == (K < 32)) ? c : (n < 32 ? s : -s);
    const unsigned off = ((n >> 3) * 8 + (K >> 3)) * 128 + (n & 7) * 16 + (K & 7) * 2;
    if constexpr (BF16) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(val);
      *reinterpret_cast<__nv_bfloat16*>(bmat + off) = hi;
      *reinterpret_cast<__nv_bfloat16*>(bmat + kTc5BBytes + off) = __float2bfloat16_rn(val - __bfloat162float(hi));
    } else {
      *reinterpret_cast<__half*>(bmat + off) = __float2half_rn(val);
    }
  }
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int k1 = e >> 5, t = e & 31;
    float s, c;
    sincospif(static_cast<float>((k1 * t) & 1023) / 512.0f, &s, &c);
    tw[e] = make_float2(c * (1.0f / 32.0f), -s * (1.0f / 32.0f));
  }
}

// Power-of-two scales of the tensor-core transforms of a mask with SLM
// energy `energy` (sum p^2) on an n x n grid: inputs times `in` stay below
// 2^15 (bound sqrt(n energy) < 2^ceil(E/2) for n energy < 2^E), outputs are
// multiplied by `out` = 32 / in. Single-precision exponent arithmetic only:
// FP64 math functions are slow on this part and this runs in every pass.
__device__ __forceinline__ void tc_scales(int n, double energy, float& in, float& out) {
  const float b2 = static_cast<float>(energy) * static_cast<float>(n);
  int E = 0;
  if (b2 > 0.f && b2 <= 3.0e38f) frexpf(b2, &E);  // b2 = f 2^E, 0.5 <= f < 1
  const int e = (E + 1) / 2 - 15;
  in = ldexpf(1.0f, -e);
  out = ldexpf(32.0f, e);
}

// Eight values as four packed pairs (FP16, or the BF16 rounded part) and, for
// BF16, the four packed pairs of their BF16 remainders.
template <bool BF16>
__device__ __forceinline__ void tc5_pack8(const float (&x)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if constexpr (BF16) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
      const float2 f = __bfloat1622float2(b);
      const __nv_bfloat162 r = __floats2bfloat162_rn(x[2 * j] - f.x, x[2 * j + 1] - f.y);
      memcpy(&h[j], &b, 4);
      memcpy(&l[j], &r, 4);
    } else {
      h[j] = tc5_pack<false>(x[2 * j], x[2 * j + 1]);
      l[j] = 0u;
    }
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

template <bool BF16>
struct Tc5Fft {
  static constexpr bool kEnabled = true;
  static constexpr bool kTcgen05 = true;
  unsigned char* abuf;  // the exchange area: half h's A operands at h * kTc5HalfStride
  unsigned bmat;        // shared-memory address of the real-form DFT matrix (BF16: hi, then lo)
  const float2* tw;     // [k1][t] twiddles / 32
  uint64_t* mbar;       // [2] completion of each half's products
  unsigned tmem;        // TMEM base of kTc5TmemCols columns
  unsigned* phase;      // this thread's parity of its half's mbarrier
  const Params* prm;    // for reporting a timeout

  // Bounded wait for this half's products; false (and GS_ETIMEOUT) if it gave up.
  __device__ __forceinline__ bool wait(int half) const {
    const bool ok = mbar_wait_bounded(&mbar[half], *phase);
    if (!ok) {
      fail(*prm, GS_ETIMEOUT);
      // give the products a second bounded period to land before the block
      // leaves and frees its TMEM
      mbar_wait_bounded(&mbar[half], *phase);
    }
    *phase ^= 1u;
    return ok;
  }

  // The transform. Every thread of the block must call it, with the same
  // scales within each half; v holds x[t + 32 i] on entry, X[t + 32 i] on exit.
  // The K-steps of one stage: A (hi, lo at +kTc5AloOffset) at a_addr with
  // step `astep` and byte offsets (lbo, sbo); B (hi, lo at +kTc5BBytes).
  __device__ __forceinline__ void issue(unsigned d_tmem, unsigned a_addr, unsigned astep, unsigned lbo, unsigned sbo,
                                        unsigned idesc) const {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const uint64_t ah = tc5_desc(a_addr + astep * s, lbo, sbo);
      const uint64_t bh = tc5_desc(bmat + 256u * s, 128u, 1024u);
      tc5_mma(d_tmem, ah, bh, idesc, s > 0 ? 1u : 0u);
      if constexpr (BF16) {
        tc5_mma(d_tmem, ah, tc5_desc(bmat + kTc5BBytes + 256u * s, 128u, 1024u), idesc, 1u);
        tc5_mma(d_tmem, tc5_desc(a_addr + kTc5AloOffset + astep * s, lbo, sbo), bh, idesc, 1u);
      }
    }
  }

  __device__ __forceinline__ void run(float2 (&v)[32], float in_scale, float out_scale) const {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = warp >> 2, wq = warp & 3;
    unsigned char* A = abuf + half * kTc5HalfStride;
    const unsigned a_addr = smem_u32(A);
    const unsigned d_tmem = tmem + 64u * half;
    const unsigned t_addr = d_tmem + (static_cast<unsigned>(32 * wq) << 16);
    const bool leader = (wq == 0) && (lane == 0);
    const int r = 32 * wq + lane;  // this thread's row of the half's product
    // the operands overwrite the half's exchange buffers: every warp of the
    // half is done with its own first
    asm volatile("bar.sync %0, 128;" ::"r"(1 + half) : "memory");
    // stage 1 operand, K-major: re x_i at K = i, im x_i at K = 32 + i
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float xr[8], xi[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        xr[j] = v[8 * c + j].x * in_scale;
        xi[j] = v[8 * c + j].y * in_scale;
      }
      uint4 hr, lr, hi_, li;
      tc5_pack8<BF16>(xr, hr, lr);
      tc5_pack8<BF16>(xi, hi_, li);
      const int o_re = ((r >> 3) * 8 + c) * 128 + (r & 7) * 16;
      const int o_im = ((r >> 3) * 8 + 4 + c) * 128 + (r & 7) * 16;
      *reinterpret_cast<uint4*>(A + o_re) = hr;
      *reinterpret_cast<uint4*>(A + o_im) = hi_;
      if constexpr (BF16) {
        *reinterpret_cast<uint4*>(A + kTc5AloOffset + o_re) = lr;
        *reinterpret_cast<uint4*>(A + kTc5AloOffset + o_im) = li;
      }
    }
    fence_proxy_async_smem();
    tc5_fence_before();  // this thread's earlier TMEM loads before the product that overwrites them
    asm volatile("bar.sync %0, 128;" ::"r"(1 + half) : "memory");
    if (leader) {
      tc5_fence_after();
      issue(d_tmem, a_addr, 256u, 128u, 1024u, tc5_idesc(BF16, false));
      tc5_commit(&mbar[half]);
    }
    wait(half);
    tc5_fence_after();
    // stage-1 result row (w, t): columns 0..31 re D1[k1], 32..63 im D1[k1]
    float d[64];
    {
      float q[16];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        tc5_ld16(q, t_addr + 16u * b);
#pragma unroll
        for (int j = 0; j < 16; ++j) d[16 * b + j] = q[j];
      }
      tc5_wait_ld();
    }
    // twiddle and the stage-2 operand, MN-major: K = t (re) and 32 + t (im),
    // M = 32 wq + k1; eight consecutive k1 make one 16-byte row of a core.
    const float2* twl = tw + lane;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      float zr[8], zi[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k1 = 8 * g + j;
        const float2 w = twl[32 * k1];
        const float a = d[k1], b = d[32 + k1];
        zr[j] = a * w.x - b * w.y;
        zi[j] = a * w.y + b * w.x;
      }
      const int mi = 4 * wq + g;
      uint4 hr, lr, hi_, li;
      tc5_pack8<BF16>(zr, hr, lr);
      tc5_pack8<BF16>(zi, hi_, li);
      const int o_re = ((lane >> 3) * 16 + mi) * 128 + (lane & 7) * 16;
      const int o_im = ((4 + (lane >> 3)) * 16 + mi) * 128 + (lane & 7) * 16;
      *reinterpret_cast<uint4*>(A + o_re) = hr;
      *reinterpret_cast<uint4*>(A + o_im) = hi_;
      if constexpr (BF16) {
        *reinterpret_cast<uint4*>(A + kTc5AloOffset + o_re) = lr;
        *reinterpret_cast<uint4*>(A + kTc5AloOffset + o_im) = li;
      }
    }
    fence_proxy_async_smem();
    tc5_fence_before();
    asm volatile("bar.sync %0, 128;" ::"r"(1 + half) : "memory");
    if (leader) {
      tc5_fence_after();
      issue(d_tmem, a_addr, 4096u, 2048u, 128u, tc5_idesc(BF16, true));
      tc5_commit(&mbar[half]);
    }
    wait(half);
    tc5_fence_after();
    {
      float q[16];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        tc5_ld16(q, t_addr + 16u * b);
#pragma unroll
        for (int j = 0; j < 16; ++j) d[16 * b + j] = q[j];
      }
      tc5_wait_ld();
    }
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) v[k2] = make_float2(d[k2] * out_scale, d[32 + k2] * out_scale);
  }
};

}  // namespace gsk
