// gs_fft.cuh -- register/shared-memory FFT building blocks for sm_103a.
//
// A length-n transform (n = 2^logn, 32 <= n <= 4096) is computed by a group
// of T = n/32 threads; thread t holds the 32 elements x[t + T*i], i = 0..31,
// in registers. The transform is a Stockham auto-sort FFT: a first radix-32
// stage entirely in registers, then further stages of radix 32 (and one final
// stage of radix 2..16 when log2(n) is not a multiple of 5), each preceded by
// one exchange through the group's padded shared-memory buffer. The output is
// left in registers in the same layout, in natural order.
//
// Only the forward transform (kernel exp(-2 pi i jk/n), unnormalised) is
// implemented. The inverse is obtained from it by exchanging real and
// imaginary parts before and after: swap(DFT(swap(x))) = n * IDFT(x). The
// kernels fold those swaps into the neighbouring projection code, so they cost
// nothing.
#pragma once

#include <cuda_runtime.h>

namespace gsk {

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * w for a twiddle w = (c, s) meaning c + i s.
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 w) {
  return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}

// cos(2 pi e / 32) for e = 0..8, rounded to float.
struct Cos32 {
  static constexpr float v[9] = {1.0f,
                                 9.807852507e-01f,
                                 9.238795042e-01f,
                                 8.314695954e-01f,
                                 7.071067691e-01f,
                                 5.555702448e-01f,
                                 3.826834261e-01f,
                                 1.950903237e-01f,
                                 0.0f};
};

// W_32^E = exp(-2 pi i E/32) = C - i S for 0 <= E < 16.
template <int E>
struct W32 {
  static constexpr float C = (E <= 8) ? Cos32::v[E] : -Cos32::v[16 - E];
  static constexpr float S = (E <= 8) ? Cos32::v[8 - E] : Cos32::v[E - 8];
};

// Radix-2 decimation-in-time butterfly (a, b) -> (a + w b, a - w b) with
// w = W_32^E (0 <= E < 16). Trivial factors (1, -i) cost only additions,
// (+-1 - i)/sqrt2 one addition pair less than a general factor, and the
// general case uses fused multiply-adds with a - w b = 2a - (a + w b).
template <int E>
__host__ __device__ __forceinline__ void bfly(float2& a, float2& b) {
  if constexpr (E == 0) {
    const float2 s = make_float2(a.x + b.x, a.y + b.y);
    b = make_float2(a.x - b.x, a.y - b.y);
    a = s;
  } else if constexpr (E == 8) {  // w = -i: w b = (b.y, -b.x)
    const float2 s = make_float2(a.x + b.y, a.y - b.x);
    b = make_float2(a.x - b.y, a.y + b.x);
    a = s;
  } else if constexpr (E == 4 || E == 12) {
    constexpr float c = Cos32::v[4];
    const float t1 = b.x + b.y;
    const float t2 = b.y - b.x;
    if constexpr (E == 4) {  // w b = c t1 + i c t2
      const float2 s = make_float2(fmaf(c, t1, a.x), fmaf(c, t2, a.y));
      b = make_float2(fmaf(-c, t1, a.x), fmaf(-c, t2, a.y));
      a = s;
    } else {  // w b = c t2 - i c t1
      const float2 s = make_float2(fmaf(c, t2, a.x), fmaf(-c, t1, a.y));
      b = make_float2(fmaf(-c, t2, a.x), fmaf(c, t1, a.y));
      a = s;
    }
  } else {
    constexpr float C = W32<E>::C;
    constexpr float S = W32<E>::S;
    // w b = (C b.x + S b.y) + i (C b.y - S b.x)
    const float2 s = make_float2(fmaf(C, b.x, fmaf(S, b.y, a.x)), fmaf(C, b.y, fmaf(-S, b.x, a.y)));
    b = make_float2(fmaf(2.f, a.x, -s.x), fmaf(2.f, a.y, -s.y));
    a = s;
  }
}

// One decimation-in-time stage with half-span H on an R-array (bit-reversed
// input order): for every block of 2H and k < H,
// (x[k], x[k + H]) -> (x[k] + W_{2H}^k x[k + H], x[k] - W_{2H}^k x[k + H]).
template <int R, int H>
struct DitStage {
  template <int BASE, int K>
  static __host__ __device__ __forceinline__ void k_loop(float2 (&a)[R]) {
    if constexpr (K < H) {
      bfly<K * (16 / H)>(a[BASE + K], a[BASE + K + H]);
      k_loop<BASE, K + 1>(a);
    }
  }
  template <int BASE>
  static __host__ __device__ __forceinline__ void b_loop(float2 (&a)[R]) {
    if constexpr (BASE < R) {
      k_loop<BASE, 0>(a);
      b_loop<BASE + 2 * H>(a);
    }
  }
  static __host__ __device__ __forceinline__ void run(float2 (&a)[R]) { b_loop<0>(a); }
};

template <int R, int H>
__host__ __device__ __forceinline__ void dit_all(float2 (&a)[R]) {
  if constexpr (H < R) {
    DitStage<R, H>::run(a);
    dit_all<R, 2 * H>(a);
  }
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

template <int R, int I>
__host__ __device__ __forceinline__ void bitrev_copy(float2 (&dst)[R], const float2 (&src)[R]) {
  if constexpr (I < R) {
    dst[I] = src[bitrev(I, ilog2(R))];
    bitrev_copy<R, I + 1>(dst, src);
  }
}

// In-register forward DFT of size R (power of two, 2 <= R <= 32), natural
// order in and out: bit-reversal permutation (register renaming only), then
// log2(R) radix-2 decimation-in-time stages.
template <int R>
__host__ __device__ __forceinline__ void dft(float2 (&a)[R]) {
  float2 t[R];
  bitrev_copy<R, 0>(t, a);
  dit_all<R, 1>(t);
#pragma unroll
  for (int i = 0; i < R; ++i) a[i] = t[i];
}

// Per-group state of a distributed transform of length N = 2^LOGN by
// T = N/32 threads. The geometry is a compile-time constant so that every
// register and shared-memory index folds to an immediate offset.
template <int LOGN>
struct GroupT {
  static constexpr int N = 1 << LOGN;
  static constexpr int T = N >> 5;
  static constexpr int SMEM = N + N / 32;  // padded exchange buffer (complex)
  int t;                                   // thread index in the group, 0..T-1
  int bar_id;                              // named barrier id (T > 32)
  float2* sm;                              // this group's exchange buffer
  const float2* __restrict__ tw;           // stage twiddle tables (twiddle_offset)

  __device__ __forceinline__ void sync() const {
    if constexpr (T <= 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "n"(T) : "memory");
    }
  }
};

// Twiddle tables. For the stage with Ns = 2^NSL and radix R the factors
// W_{Ns R}^{r m} (1 <= m < R, r < Ns) are stored transposed, entry
// (m - 1) * Ns + r, so that the threads of a warp (consecutive r) read
// consecutive addresses. The stage with NSL = 5 starts at entry 0; the stage
// with NSL = 10 (only for N > 1024, after a radix-32 stage) at entry 31 * 32.
__host__ __device__ constexpr int twiddle_offset(int nsl) { return nsl == 5 ? 0 : 31 * 32; }

// Twiddles of the stage that follows the first 32 points (NSL = 5), held in
// registers: thread t needs W_{32 R}^{r m} for r = (t + T b) mod 32, b < 32/R,
// 1 <= m < R. Loaded once and reused by every transform of the same length.
template <int LOGN>
struct StageTw {
  static constexpr int R = (LOGN <= 5) ? 1 : ((LOGN - 5 >= 5) ? 32 : (1 << (LOGN - 5)));
  static constexpr int Q = 32 / R;
  static constexpr int COUNT = (R > 1) ? (R - 1) * Q : 1;
  float2 w[COUNT];

  __device__ __forceinline__ void load(const float2* __restrict__ tw, int t) {
    if constexpr (R > 1) {
      constexpr int T = (1 << LOGN) >> 5;
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        const int r = (t + T * b) & 31;
#pragma unroll
        for (int m = 1; m < R; ++m) w[b * (R - 1) + m - 1] = __ldg(tw + (m - 1) * 32 + r);
      }
    }
  }
};

// Stockham stage of radix R with Ns = 2^NSL: butterflies j = t + T*b,
// b < 32/R. Butterfly j reads x[j + m N/R] = v[b + (32/R) m], multiplies by
// W_{Ns R}^{(j mod Ns) m} and transforms over m; for the last stage the
// outputs land at the same register positions.
template <int LOGN, int NSL, int R>
__device__ __forceinline__ void stage_c(float2 (&v)[32], const GroupT<LOGN>& g, const StageTw<LOGN>& sw) {
  constexpr int Q = 32 / R;
  constexpr int T = GroupT<LOGN>::T;
  constexpr int NS = 1 << NSL;
#pragma unroll
  for (int b = 0; b < Q; ++b) {
    float2 a[R];
#pragma unroll
    for (int m = 0; m < R; ++m) a[m] = v[b + Q * m];
    if constexpr (NSL == 5) {
#pragma unroll
      for (int m = 1; m < R; ++m) a[m] = cmul(a[m], sw.w[b * (R - 1) + m - 1]);
    } else if constexpr (NSL > 0) {
      const int r = (g.t + T * b) & (NS - 1);
      const float2* __restrict__ w = g.tw + twiddle_offset(NSL) + r;
#pragma unroll
      for (int m = 1; m < R; ++m) a[m] = cmul(a[m], __ldg(w + (m - 1) * NS));
    }
    dft<R>(a);
#pragma unroll
    for (int m = 0; m < R; ++m) v[b + Q * m] = a[m];
  }
}

// Exchange after a radix-32 stage with Ns = 2^NSL (butterfly j = t): output
// m goes to (t / Ns) 32 Ns + (t mod Ns) + m Ns; then every thread reads back
// x[t + T i]. Index i of the padded buffer lives at i + i/32.
template <int LOGN, int NSL>
__device__ __forceinline__ void exchange(float2 (&v)[32], const GroupT<LOGN>& g) {
  constexpr int T = GroupT<LOGN>::T;
  static_assert(NSL == 0 || NSL >= 5, "exchanges follow radix-32 stages");
  if constexpr (NSL == 0) {
    float2* w = g.sm + 33 * g.t;
#pragma unroll
    for (int m = 0; m < 32; ++m) w[m] = v[m];
  } else {
    const int base = ((g.t >> NSL) << (NSL + 5)) + (g.t & ((1 << NSL) - 1));
    float2* w = g.sm + base + (base >> 5);
    constexpr int STR = (1 << NSL) + (1 << (NSL - 5));
#pragma unroll
    for (int m = 0; m < 32; ++m) w[m * STR] = v[m];
  }
  g.sync();
  if constexpr (T >= 32) {
    const float2* r = g.sm + g.t + (g.t >> 5);
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = r[i * (T + T / 32)];
  } else {
    const float2* r = g.sm + g.t;
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = r[i * T + ((i * T) >> 5)];
  }
  g.sync();
}

template <int LOGN, int DONE>
__device__ __forceinline__ void fft_from(float2 (&v)[32], const GroupT<LOGN>& g, const StageTw<LOGN>& sw) {
  if constexpr (DONE < LOGN) {
    if constexpr (DONE > 0) exchange<LOGN, DONE - 5>(v, g);
    constexpr int REM = LOGN - DONE;
    constexpr int RL = REM >= 5 ? 5 : REM;
    stage_c<LOGN, DONE, (1 << RL)>(v, g, sw);
    fft_from<LOGN, DONE + RL>(v, g, sw);
  }
}

// Forward unnormalised DFT of length N over the group: v holds x[t + T i] on
// entry and X[t + T i] on exit. Every thread of the group must call it.
template <int LOGN>
__device__ __forceinline__ void group_fft(float2 (&v)[32], const GroupT<LOGN>& g, const StageTw<LOGN>& sw) {
  fft_from<LOGN, 0>(v, g, sw);
}

}  // namespace gsk
