// gs_tc5.cuh -- the DFTs of the tensor-core form on the fifth-generation
// tensor cores (tcgen05): FP16 or BF16 operands in shared memory, FP32
// accumulators in tensor memory (TMEM), for lines of n = 32 R points
// (R = 8, 16, 32: the square grids 256, 512, 1024).
//
// Same arithmetic as gs_tc.cuh (the four-step factorisation n = 32 x R, both
// stages dense products with the real forms of the 32-point and R-point DFT
// matrices), but batched over the four warps of one half of the block. Lane
// l = R gamma + t of a warp holds x_gamma[t + R i], i = 0..31, of line gamma
// of the warp (32/R lines per warp: the thread layout of the FP32
// transforms). Each stage is issued by one thread of the half:
//
//   stage 1  D1[(w, l)][k1] = sum_i x[t + R i] W_32^{i k1}          one M = 128 product, N = K = 64
//            (A K-major: row (w, l) = [re x_i | im x_i])
//   twiddle  Z[(gamma, k1)][t] = D1[(w, l)][k1] W_n^{k1 t} / 32      (epilogue of tcgen05.ld, FP32)
//   stage 2  D2[(gamma, k1)][k2] = sum_t Z[(gamma, k1)][t] W_R^{t k2}   32/R products, M = 128, N = K = 2R
//            (A MN-major: column t = [re | im])
//            X_gamma[k1 + 32 k2] = 32 D2[(gamma, k1)][k2]
//
// The rows of stage 2 are placed so that every lane reads back its own
// outputs: row (gamma, k1) of warp w goes to tile c = k1 / R (its own
// product, 2R TMEM columns) at TMEM lane 32 (w mod 4) + R gamma + (k1 mod R),
// so lane R gamma + t finds rows (gamma, t + R c), i.e. X_gamma[t + R (c +
// (32/R) k2)], in its own lane of every tile: the result lands in the thread
// layout the transform started from, with no exchange. Stage 1 of every
// length uses the same 64 TMEM columns per half as stage 2 ((32/R) tiles of
// 2R columns), and four tcgen05.mma (K = 16 each) per half and stage. The two
// halves of the block run their products independently (own mbarrier, own
// TMEM columns, own named barrier), so one half's tensor-core latency can
// overlap the other's FP32 epilogue.
//
// Shared-memory operands use the canonical no-swizzle layout: 8 x 16-byte
// core matrices, 128 bytes each. K-major: core (m/8, k/8) at ((m/8) (K/8) +
// k/8) 128, row m mod 8 at 16 (m mod 8); the leading byte offset (next core
// along K) is 128, the stride byte offset (next core along M or N) (K/8) 128.
// MN-major: core (m/8, k/8) at ((k/8) 16 + m/8) 128 within an M-tile of 128
// rows, row k mod 8 at 16 (k mod 8), m mod 8 at 2 (m mod 8); leading byte
// offset (along K) 2048, stride byte offset (along M) 128.
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
// the real-form 32-point DFT matrix B1, the real-form R-point matrix B2 (each
// its FP16 or BF16 rounding, then for BF16 the remainder: tc5_real_form) and
// the 8 KiB twiddle table [k1][lane]. The A operands live in the exchange
// area (kTc5HalfStride bytes per half: A_hi 16 KiB, A_lo 16 KiB).
constexpr int kTc5HalfStride = 4 * 32 * 33 * 8;  // the exchange buffers of four warps
constexpr int kTc5AloOffset = 16384;
constexpr int kTc5BBytes = 64 * 64 * 2;          // one real-form matrix of the largest size, one part
constexpr int kTc5B2Offset = 2 * kTc5BBytes;
constexpr int kTc5TwOffset = 4 * kTc5BBytes;
constexpr int kTc5TwBytes = 32 * 32 * 8;
constexpr int kTc5SmemBytes = 4 * kTc5BBytes + kTc5TwBytes;
// bytes of one part of the real form of the P-point DFT matrix (2P x 2P)
__host__ __device__ constexpr int tc5_form_bytes(int P) { return 2 * P * 2 * P * 2; }
static_assert(kTc5SmemBytes == kTc5ExtraSmemBytes, "tcgen05 tables match the launch size");
static_assert(2 * kTc5AloOffset <= kTc5HalfStride, "both A operands of a half fit its exchange buffers");
constexpr int kTc5TmemCols = 128;  // two halves x 64 FP32 columns

__device__ __forceinline__ uint64_t tc5_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (static_cast<uint64_t>(1) << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, FP16 (0) or BF16 (1)
// operands, A K-major (0) or MN-major (1), B K-major, N columns, M = 128.
__host__ __device__ constexpr unsigned tc5_idesc(bool bf16, bool a_mn, unsigned n) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((a_mn ? 1u : 0u) << 15) |
         ((n >> 3) << 17) | ((128u >> 4) << 24);
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

// The real form of the P-point DFT matrix (P = 32 or R) as a K-major B
// operand of 2P x 2P at dst (remainder at dst + tc5_form_bytes(P) for BF16): row n
// < P gives Re y_n, n >= P gives Im y_{n-P}; column K < P multiplies re x_K,
// K >= P im x_{K-P}:
//   B[n][K] = cos, B[n][P+K] = sin, B[P+n][K] = -sin, B[P+n][P+K] = cos
// of 2 pi n K / P (since W (a + i b) = (c a + s b) + i (c b - s a) for
// W = c - i s).
template <int P, bool BF16>
__device__ void tc5_real_form(unsigned char* dst) {
  constexpr int P2 = 2 * P;
  for (int e = threadIdx.x; e < P2 * P2; e += blockDim.x) {
    const int n = e / P2, K = e % P2;
    const int kk = K % P, nn = n % P;
    float s, c;
    sincospif(2.0f * static_cast<float>((nn * kk) % P) / static_cast<float>(P), &s, &c);
    const float val = ((n < P) == (K < P)) ? c : (n < P ? s : -s);
    const unsigned off = ((n >> 3) * (P2 / 8) + (K >> 3)) * 128 + (n & 7) * 16 + (K & 7) * 2;
    if constexpr (BF16) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(val);
      *reinterpret_cast<__nv_bfloat16*>(dst + off) = hi;
      *reinterpret_cast<__nv_bfloat16*>(dst + tc5_form_bytes(P) + off) =
          __float2bfloat16_rn(val - __bfloat162float(hi));
    } else {
      *reinterpret_cast<__half*>(dst + off) = __float2half_rn(val);
    }
  }
}

// The block's constant tables for lines of n = 2^LOGN: B1 (32-point, unless
// b1 is null: shared by every length), B2 (R-point) and the stage twiddles
// tw[k1][lane] = W_n^{k1 t} / 32 with t = lane mod R.
template <int LOGN, bool BF16>
__device__ void tc5_build_tables(unsigned char* b1, unsigned char* b2, float2* tw) {
  constexpr int N = 1 << LOGN;
  constexpr int R = N >> 5;
  if (b1 != nullptr) tc5_real_form<32, BF16>(b1);
  tc5_real_form<R, BF16>(b2);
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int k1 = e >> 5, t = (e & 31) & (R - 1);
    float s, c;
    sincospif(2.0f * static_cast<float>((k1 * t) % N) / static_cast<float>(N), &s, &c);
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

template <int LOGN, bool BF16>
struct Tc5Fft {
  static constexpr bool kEnabled = true;
  static constexpr bool kTcgen05 = true;
  static constexpr int N = 1 << LOGN;
  static constexpr int R = N >> 5;   // stage-2 length
  static constexpr int Q = 32 / R;   // lines per warp = stage-2 tiles per half
  static constexpr int N2 = 2 * R;   // stage-2 N and K (real form)
  static_assert(R == 8 || R == 16 || R == 32, "tcgen05 transforms have length 256, 512 or 1024");
  unsigned char* abuf;  // the exchange area: half h's A operands at h * kTc5HalfStride
  unsigned b1, b2;      // shared-memory addresses of the real-form matrices (tc5_build_tables)
  const float2* tw;     // [k1][lane] twiddles / 32
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

  // The K-steps of one product into d_tmem: A (hi, lo at +kTc5AloOffset) at
  // a_addr with step `astep` and byte offsets (lbo, sbo); B (hi, lo at
  // +b_lo) at b_addr, K-major with stride byte offset b_sbo.
  template <int KSTEPS>
  __device__ __forceinline__ void issue(unsigned d_tmem, unsigned a_addr, unsigned astep, unsigned lbo, unsigned sbo,
                                        unsigned b_addr, unsigned b_sbo, unsigned b_lo, unsigned idesc) const {
#pragma unroll
    for (int s = 0; s < KSTEPS; ++s) {
      const uint64_t ah = tc5_desc(a_addr + astep * s, lbo, sbo);
      const uint64_t bh = tc5_desc(b_addr + 256u * s, 128u, b_sbo);
      tc5_mma(d_tmem, ah, bh, idesc, s > 0 ? 1u : 0u);
      if constexpr (BF16) {
        tc5_mma(d_tmem, ah, tc5_desc(b_addr + b_lo + 256u * s, 128u, b_sbo), idesc, 1u);
        tc5_mma(d_tmem, tc5_desc(a_addr + kTc5AloOffset + astep * s, lbo, sbo), bh, idesc, 1u);
      }
    }
  }

  // The transform. Every thread of the half must call it, with the same
  // scales; v holds x[t + R i] on entry, X[t + R i] on exit (lane R gamma + t).
  __device__ __forceinline__ void run(float2 (&v)[32], float in_scale, float out_scale) const {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = warp >> 2, wq = warp & 3;
    const int gam = lane / R, t = lane & (R - 1);
    unsigned char* A = abuf + half * kTc5HalfStride;
    const unsigned a_addr = smem_u32(A);
    const unsigned d_tmem = tmem + 64u * half;
    const unsigned t_addr = d_tmem + (static_cast<unsigned>(32 * wq) << 16);
    const bool leader = (wq == 0) && (lane == 0);
    const int r = 32 * wq + lane;  // this thread's row of the half's stage-1 product
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
      issue<4>(d_tmem, a_addr, 256u, 128u, 1024u, b1, 1024u, tc5_form_bytes(32), tc5_idesc(BF16, false, 64u));
      tc5_commit(&mbar[half]);
    }
    wait(half);
    tc5_fence_after();
    // stage-1 result row (w, lane): columns 0..31 re D1[k1], 32..63 im D1[k1]
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
    // twiddle and the stage-2 operand, MN-major: K = t (re) and R + t (im);
    // row (gamma, k1) in tile c = k1 / R at M = 32 wq + R gamma + (k1 mod R),
    // so eight consecutive k1 make one 16-byte row of a core
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
      const int c = (8 * g) / R;
      const int m = 32 * wq + R * gam + (8 * g) % R;
      uint4 hr, lr, hi_, li;
      tc5_pack8<BF16>(zr, hr, lr);
      tc5_pack8<BF16>(zi, hi_, li);
      const int tile = c * R * 512;  // (2R/8) k-cores of 16 m-cores of 128 bytes
      const int o_re = tile + ((t >> 3) * 16 + (m >> 3)) * 128 + (t & 7) * 16;
      const int o_im = tile + (((R + t) >> 3) * 16 + (m >> 3)) * 128 + ((R + t) & 7) * 16;
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
#pragma unroll
      for (int c = 0; c < Q; ++c)
        issue<N2 / 16>(d_tmem + static_cast<unsigned>(c * N2), a_addr + c * R * 512, 4096u, 2048u, 128u, b2,
                       (N2 / 8) * 128u, tc5_form_bytes(R), tc5_idesc(BF16, true, N2));
      tc5_commit(&mbar[half]);
    }
    wait(half);
    tc5_fence_after();
    {
      float q[16];
#pragma unroll
      for (int c = 0; c < Q; ++c) {
#pragma unroll
        for (int b = 0; b < N2 / 16; ++b) {
          tc5_ld16(q, t_addr + static_cast<unsigned>(c * N2 + 16 * b));
#pragma unroll
          for (int j = 0; j < 16; ++j) d[c * N2 + 16 * b + j] = q[j];
        }
      }
      tc5_wait_ld();
    }
    // tile c holds re X[t + R (c + Q k2)] in columns k2 < R, im in R + k2
#pragma unroll
    for (int c = 0; c < Q; ++c)
#pragma unroll
      for (int k2 = 0; k2 < R; ++k2)
        v[c + Q * k2] = make_float2(d[c * N2 + k2] * out_scale, d[c * N2 + R + k2] * out_scale);
  }
};

}  // namespace gsk
