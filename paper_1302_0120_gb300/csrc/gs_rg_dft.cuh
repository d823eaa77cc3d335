// gs_rg_dft.cuh -- DFTs of compile-time length held in one thread's registers,
// for the register-resident general-grid kernel (gs_rg.cuh).
//
// rdft<N> transforms a[0..N) in place, natural order in and out, unnormalised,
// kernel exp(-2 pi i jk/N), for 5-smooth N up to 32. Powers of two use the
// radix-2 code of gs_fft.cuh, 3 and 5 the kernels of gs_general.cuh; any other
// N = P Q is one Cooley-Tukey step in registers (decimation in time):
//
//   n = r + P s (r < P, s < Q),  k = k1 + Q j (k1 < Q, j < P)
//   X[k1 + Q j] = sum_r W_P^{r j} W_N^{r k1} sum_s a[r + P s] W_Q^{s k1}
//
// so P sub-DFTs of length Q, the twiddles W_N^{r k1}, then Q DFTs of length P.
// Every index is a compile-time constant and every twiddle an immediate: the
// twiddles are evaluated by the compiler (unit_cs) in double and rounded once
// to float.
#pragma once

#include <type_traits>

#include "gs_fft.cuh"
#include "gs_general.cuh"

namespace gsk {

// cos and sin of 2 pi m / n, evaluated in double at compile time: the angle
// is reduced exactly, in integers, to [0, pi/4] by the symmetries of the
// circle (u -> 1 - u, u -> 1/2 - u, u -> 1/4 - u for u = m/n turns), then the
// Taylor series of cos and sin about 0 are summed to the x^23 term (truncation
// below 1e-20 on [0, pi/4]).
struct CosSin {
  double c, s;
};

__host__ __device__ constexpr CosSin taylor_cos_sin(double x) {
  double c = 1.0, s = x, tc = 1.0, ts = x;
  for (int k = 1; k <= 11; ++k) {
    tc *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    ts *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    c += tc;
    s += ts;
  }
  return CosSin{c, s};
}

__host__ __device__ constexpr CosSin unit_cs(long long m, long long n) {
  constexpr double kTwoPi = 6.283185307179586476925286766559;
  m %= n;
  if (m < 0) m += n;
  long long num = m, den = n;  // u = num / den turns
  bool neg_s = false, neg_c = false, swap = false;
  if (2 * num > den) {  // cos(2 pi u) = cos(2 pi (1 - u)), sin negated
    num = den - num;
    neg_s = true;
  }
  if (4 * num > den) {  // u in (1/4, 1/2]: cos(2 pi u) = -cos(2 pi (1/2 - u)), sin kept
    num = den - 2 * num;
    den *= 2;
    neg_c = true;
  }
  if (8 * num > den) {  // u in (1/8, 1/4]: cos and sin of 2 pi (1/4 - u), exchanged
    num = den - 4 * num;
    den *= 4;
    swap = true;
  }
  CosSin r = taylor_cos_sin(kTwoPi * static_cast<double>(num) / static_cast<double>(den));
  if (swap) r = CosSin{r.s, r.c};
  if (neg_c) r.c = -r.c;
  if (neg_s) r.s = -r.s;
  return r;
}

// x * W_N^E = x * exp(-2 pi i E/N), the factor an immediate.
template <int N, int E>
__host__ __device__ __forceinline__ float2 twmul(float2 x) {
  constexpr CosSin w = unit_cs(E, N);
  constexpr float c = static_cast<float>(w.c);
  constexpr float s = static_cast<float>(w.s);
  // (x.x + i x.y)(c - i s)
  return make_float2(fmaf(x.x, c, x.y * s), fmaf(x.y, c, -(x.x * s)));
}

// f(integral_constant<int, I>) for I = B .. E-1, unrolled at compile time.
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// First factor P of the Cooley-Tukey step for length N (the sub-DFTs of
// length Q = N / P are then the longer ones).
__host__ __device__ constexpr int rdft_split(int n) {
  return (n % 5 == 0 && n > 5) ? 5 : (n % 3 == 0 && n > 3) ? 3 : (n % 4 == 0 && n > 4) ? 4 : 2;
}

__host__ __device__ constexpr bool is_pow2_c(int n) { return n > 0 && (n & (n - 1)) == 0; }

template <int N>
__host__ __device__ __forceinline__ void rdft(float2 (&a)[N]) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (is_pow2_c(N)) {
    dft<N>(a);
  } else if constexpr (N == 3) {
    dft3(a);
  } else if constexpr (N == 5) {
    dft5(a);
  } else {
    constexpr int P = rdft_split(N);
    constexpr int Q = N / P;
    static_assert(P * Q == N, "5-smooth lengths only");
    float2 b[P][Q];
#pragma unroll
    for (int r = 0; r < P; ++r) {
#pragma unroll
      for (int s = 0; s < Q; ++s) b[r][s] = a[r + P * s];
      rdft<Q>(b[r]);
    }
    static_for<1, P>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      static_for<1, Q>([&](auto kc) {
        constexpr int k1 = decltype(kc)::value;
        b[r][k1] = twmul<N, r * k1>(b[r][k1]);
      });
    });
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) {
      float2 c[P];
#pragma unroll
      for (int r = 0; r < P; ++r) c[r] = b[r][k1];
      rdft<P>(c);
#pragma unroll
      for (int j = 0; j < P; ++j) a[k1 + Q * j] = c[j];
    }
  }
}

}  // namespace gsk
