// gs_tc.cuh -- a warp-level DFT of length n = 32 R (R = 8, 16, 32) on the
// tensor cores, with FP16 operands and FP32 accumulation.
//
// The transform has the same interface as group_fft: on entry lane
// l = gamma R + t holds x_gamma[t + R i] (i = 0..31) of transform gamma
// (32/R transforms per warp), on exit it holds X_gamma[t + R i], unnormalised,
// exp(-2 pi i jk/n). It is the four-step factorisation n = 32 x R written as
// two dense complex matrix products:
//
//   stage 1  Y[k1][t]  = sum_i  F32[k1][i] x[t + R i]          (k1, i < 32)
//   twiddle  Z[k1][t]  = Y[k1][t] W_n^{k1 t} / 32
//   stage 2  X[k1 + 32 k2] = 32 sum_t FR[k2][t] Z[k1][t]        (k2, t < R)
//
// Each complex product is one real product with the real form
// [[Fr, -Fi], [Fi, Fr]] of the DFT matrix and the operand stacked as
// [re; im], issued as mma.sync m16n8k16 tiles (row-major A = DFT matrix,
// column-major B = data). The DFT-matrix fragments stay in registers for the
// whole kernel; the stage-1 operand is staged in the warp's shared-memory
// buffer as FP16 and read with ldmatrix; the stage-1 result, twiddled and
// rounded to FP16, feeds stage 2 from registers (its accumulator tiles are
// the transposed B operand of stage 2); the stage-2 result (FP32) returns to
// the thread layout through the buffer. The factor 1/32 before the FP16
// rounding of Z and the exact factor 32 after stage 2 are powers of two.
//
// Range: every FP16 value is at most max |x| in magnitude; the caller scales
// the inputs by a power of two that keeps them below 2^15 (and the outputs
// back). Rounding: unit roundoff 2^-11 per FP16 operand; the relative L2
// error of one transform is about 3e-4.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>

#include "gs_fft.cuh"
#include "gs_tma.cuh"

namespace gsk {

// Per-warp buffer: 32 x 33 complex (8448 bytes), the same slice of shared
// memory that the thread groups of that warp use for their FFT exchanges.
constexpr int kTcWarpBytes = 32 * 33 * 8;
// Stage twiddles of the block: [32 slots][32 lanes] complex, then the table
// (cos, sin)(2 pi e / 32), e < 32.
constexpr int kTcTwBytes = 32 * 32 * 8;
constexpr int kTcCsBytes = 32 * 8;

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p))
               : "memory");
}

// Fill the block's tables: cs[e] = (cos, sin)(2 pi e/32) and, for the
// stage-1 result element `slot` of lane l, tw[slot * 32 + l] = W_n^{k1 t}/32.
// Slot = ((mp * 4 + nt) * 2 + h) * 2 + e holds row k1 = 16 mp + 8 h + l/4 and
// column j = 8 nt + 2 (l mod 4) + e of the stage-1 product, t = j mod R.
template <int LOGN>
__device__ void tc_build_tables(float2* tw, float2* cs) {
  constexpr int N = 1 << LOGN;
  constexpr int R = N >> 5;
  for (int e = threadIdx.x; e < 32 * 32 + 32; e += blockDim.x) {
    float s, c;
    if (e < 32 * 32) {
      const int lane = e & 31;
      const int slot = e >> 5;
      const int k1 = 16 * (slot >> 4) + 8 * ((slot >> 1) & 1) + (lane >> 2);
      const int t = (8 * ((slot >> 2) & 3) + 2 * (lane & 3) + (slot & 1)) % R;
      sincospif(2.0f * static_cast<float>((k1 * t) % N) / static_cast<float>(N), &s, &c);
      tw[e] = make_float2(c * (1.0f / 32.0f), -s * (1.0f / 32.0f));
    } else {
      sincospif(static_cast<float>(e - 32 * 32) / 16.0f, &s, &c);
      cs[e - 32 * 32] = make_float2(c, s);
    }
  }
}

// Element (row r, column k) of the real form [[C, S], [-S, C]] of the
// R-point DFT matrix (C = cos, S = sin of 2 pi k2 t / R; rows k2 + R rb,
// columns t + R kb), in FP32 from the block's cos/sin table.
template <int R>
__device__ __forceinline__ float real_form(const float2* cs, int r, int k) {
  const int rb = r / R, kb = k / R;
  const int e = ((r % R) * (k % R) * (32 / R)) & 31;
  const float2 w = cs[e];
  return rb == kb ? w.x : (rb == 0 ? w.y : -w.y);
}

// The four registers of the A fragment of the 16 x 16 tile (mt, kt) of a
// real-form matrix, for this lane.
template <int R>
__device__ __forceinline__ void a_tile(uint32_t (&a)[4], const float2* cs, int mt, int kt) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, c = lane & 3;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = 16 * mt + g + 8 * (q & 1);
    const int k = 16 * kt + 2 * c + 8 * (q >> 1);
    a[q] = pack_h2(real_form<R>(cs, r, k), real_form<R>(cs, r, k + 1));
  }
}

// Stage-1 fragments, the same for every transform length: the 32-point real
// form [[C, S], [-S, C]] from its 16 x 16 sub-tiles of C, S and -S (tile
// (mt, kt) of the 64 x 64 matrix), held in registers for a whole launch.
struct TcStage1 {
  uint32_t fc[2][2][4], fs[2][2][4], fn[2][2][4];

  __device__ __forceinline__ void load(const float2* cs) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        a_tile<32>(fc[a][b], cs, a, b);      // rows 0..31, columns 0..31: C
        a_tile<32>(fs[a][b], cs, a, 2 + b);  // rows 0..31, columns 32..63: S
        a_tile<32>(fn[a][b], cs, 2 + a, b);  // rows 32..63, columns 0..31: -S
      }
  }

  // C/D += tile (mt, kt) of the 32-point real form times B.
  __device__ __forceinline__ void mma32(float (&d)[4], int mt, int kt, uint32_t b0, uint32_t b1) const {
    const int a = mt & 1, b = kt & 1;
    if ((mt >> 1) == (kt >> 1)) mma_16816(d, fc[a][b], b0, b1);
    else if ((mt >> 1) == 0) mma_16816(d, fs[a][b], b0, b1);
    else mma_16816(d, fn[a][b], b0, b1);
  }
};

// Stage-2 fragments of the R-point real form for R < 32 (R = 32 reuses
// stage 1's).
template <int R>
struct TcStage2 {
  static constexpr int KT = R / 8;
  uint32_t fr[KT][KT][4];
  __device__ __forceinline__ void load(const float2* cs) {
#pragma unroll
    for (int mt = 0; mt < KT; ++mt)
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) a_tile<R>(fr[mt][kt], cs, mt, kt);
  }
};

template <>
struct TcStage2<32> {
  __device__ __forceinline__ void load(const float2*) {}
};

// The transform of length 2^LOGN: a view of the launch's fragments and of
// this length's stage twiddles in shared memory.
template <int LOGN>
struct TcFft {
  static constexpr bool kEnabled = true;
  static constexpr bool kTcgen05 = false;
  static constexpr int N = 1 << LOGN;
  static constexpr int R = N >> 5;
  static constexpr int Q = 32 / R;       // transforms per warp
  static constexpr int KT = R / 8;       // 16-wide tiles along 2R
  static constexpr int XS = 72;          // halves per row of the stage-1 operand (144 bytes)
  static_assert(R == 8 || R == 16 || R == 32, "tensor-core transforms have length 256, 512 or 1024");
  static_assert(Q * (N + 8) <= 32 * 33 && 32 * XS * 2 <= kTcWarpBytes, "buffers fit the warp slice");

  const TcStage1& s1;
  const TcStage2<R>& s2;
  const float2* tw;  // stage twiddles of this length (tc_build_tables)

  // C/D += tile (mt, kt) of the stage-2 real form times B.
  __device__ __forceinline__ void mma2(float (&d)[4], int mt, int kt, uint32_t b0, uint32_t b1) const {
    if constexpr (R == 32) s1.mma32(d, mt, kt, b0, b1);
    else mma_16816(d, s2.fr[mt][kt], b0, b1);
  }

  // Position of element j of transform gamma in the FP32 return buffer; the
  // XOR keeps both the fragment-order writes and the thread-order reads free
  // of bank conflicts.
  __device__ static __forceinline__ int pos(int gamma, int j) {
    const int k2 = j >> 5;
    return gamma * (N + 8) + (k2 << 5) + ((j & 31) ^ ((k2 & 1) | ((k2 & 2) << 2)));
  }

  // The transform. `buf` is the warp's 16-byte aligned slice (kTcWarpBytes).
  // Every lane of the warp must call it. The inputs are multiplied by the
  // power of two `in_scale` before the FP16 rounding and the outputs by
  // `out_scale` (32 / in_scale: the 1/32 in the twiddles is undone as well).
  __device__ __forceinline__ void run(float2 (&v)[32], unsigned char* buf, float in_scale, float out_scale) const {
    const int lane = threadIdx.x & 31;
    __half* xs = reinterpret_cast<__half*>(buf);
    // Stage-1 operand B: row n = lane holds re x[.. i ..] at column i, im at 32 + i.
    {
      uint4* row = reinterpret_cast<uint4*>(xs + lane * XS);
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = make_float2(v[i].x * in_scale, v[i].y * in_scale);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        row[c] = make_uint4(pack_h2(v[8 * c].x, v[8 * c + 1].x), pack_h2(v[8 * c + 2].x, v[8 * c + 3].x),
                            pack_h2(v[8 * c + 4].x, v[8 * c + 5].x), pack_h2(v[8 * c + 6].x, v[8 * c + 7].x));
        row[4 + c] = make_uint4(pack_h2(v[8 * c].y, v[8 * c + 1].y), pack_h2(v[8 * c + 2].y, v[8 * c + 3].y),
                                pack_h2(v[8 * c + 4].y, v[8 * c + 5].y), pack_h2(v[8 * c + 6].y, v[8 * c + 7].y));
      }
    }
    __syncwarp();
    float acc[4][4][4];  // [mt][nt][reg]; mt 0, 1: real rows, 2, 3: imaginary rows
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      uint32_t b[2][4];
      const __half* src = xs + (8 * nt + (lane & 7)) * XS + 8 * (lane >> 3);
      ldsm_x4(b[0], src);
      ldsm_x4(b[1], src + 32);
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) s1.mma32(acc[mt][nt], mt, kt, b[kt >> 1][2 * (kt & 1)], b[kt >> 1][2 * (kt & 1) + 1]);
    }
    // Twiddle, 1/32, FP16. The stage-2 operand B of transform gamma (K = t,
    // re then im; N = k1) is the transpose of the stage-1 accumulator (rows
    // k1, re then im; columns gamma R + t), so this lane's pair of adjacent
    // columns of an 8-column accumulator tile is exactly a B register: the
    // packed values stay in registers. z[part][nt][mp][h]: part 0 re, 1 im;
    // rows k1 = 16 mp + 8 h + g, columns 8 nt + 2c, 8 nt + 2c + 1.
    uint32_t z[2][4][2][2];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int mp = 0; mp < 2; ++mp)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int slot = ((mp * 4 + nt) * 2 + h) * 2;
          const float2 w0 = tw[slot * 32 + lane];
          const float2 w1 = tw[(slot + 1) * 32 + lane];
          const float2 y0 = cmul(make_float2(acc[mp][nt][2 * h], acc[mp + 2][nt][2 * h]), w0);
          const float2 y1 = cmul(make_float2(acc[mp][nt][2 * h + 1], acc[mp + 2][nt][2 * h + 1]), w1);
          z[0][nt][mp][h] = pack_h2(y0.x, y1.x);
          z[1][nt][mp][h] = pack_h2(y0.y, y1.y);
        }

    // Stage 2 per transform: tiles [gamma][mt][nt], mt < KT (R = 32: mt 0, 1
    // real rows, 2, 3 imaginary rows). B tile (kt, nt) holds rows k = 16 kt
    // + 2c (+1) in b0 and k + 8 in b1, row k being re Z[.][k] for k < R and
    // im Z[.][k - R] otherwise, at columns k1 = 8 nt + g.
    float out[Q][KT][4][4];
#pragma unroll
    for (int gamma = 0; gamma < Q; ++gamma)
#pragma unroll
      for (int mt = 0; mt < KT; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q) out[gamma][mt][nt][q] = 0.f;
#pragma unroll
    for (int gamma = 0; gamma < Q; ++gamma) {
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
          const int ka = 16 * kt, kb = 16 * kt + 8;  // first rows of b0 and b1
          const uint32_t b0 = z[ka < R ? 0 : 1][(gamma * R + ka % R) >> 3][nt >> 1][nt & 1];
          const uint32_t b1 = z[kb < R ? 0 : 1][(gamma * R + kb % R) >> 3][nt >> 1][nt & 1];
#pragma unroll
          for (int mt = 0; mt < KT; ++mt) mma2(out[gamma][mt][nt], mt, kt, b0, b1);
        }
      }
    }
    __syncwarp();  // operand reads done before the return buffer overwrites them

    // Back to the thread layout through the FP32 buffer, times 32.
    float2* ret = reinterpret_cast<float2*>(buf);
    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int gamma = 0; gamma < Q; ++gamma)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int k1 = 8 * nt + 2 * c + e;
          if constexpr (R == 32) {
#pragma unroll
            for (int mp = 0; mp < 2; ++mp)
#pragma unroll
              for (int h = 0; h < 2; ++h)
                ret[pos(0, k1 + 32 * (16 * mp + 8 * h + g))] =
                    make_float2(out_scale * out[0][mp][nt][2 * h + e], out_scale * out[0][mp + 2][nt][2 * h + e]);
          } else if constexpr (R == 16) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
              ret[pos(gamma, k1 + 32 * (8 * h + g))] =
                  make_float2(out_scale * out[gamma][0][nt][2 * h + e], out_scale * out[gamma][1][nt][2 * h + e]);
          } else {
            ret[pos(gamma, k1 + 32 * g)] =
                make_float2(out_scale * out[gamma][0][nt][e], out_scale * out[gamma][0][nt][2 + e]);
          }
        }
    __syncwarp();
    const int gl = lane / R, tl = lane % R;
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = ret[pos(gl, tl + R * i)];
    __syncwarp();  // the caller may reuse the buffer
  }
};

}  // namespace gsk
