// Host-side check of the register DFTs of the general-grid kernel
// (paper_1302_0120_gb300/csrc/gs_rg_dft.cuh): rdft<N> against the direct DFT
// summed in double, and the compiler-evaluated cos/sin (unit_cs) against the
// C library. Built with nvcc as host code by tests/test_rdft_host.py; prints
// one line per check, "N err" or "cs err".
#include <cmath>
#include <cstdio>
#include <random>

#include "gs_rg_dft.cuh"

template <int N>
static double check() {
  std::mt19937 g(N);
  std::uniform_real_distribution<float> u(-1.f, 1.f);
  float2 a[N];
  double xr[N], xi[N];
  for (int i = 0; i < N; ++i) {
    a[i] = make_float2(u(g), u(g));
    xr[i] = a[i].x;
    xi[i] = a[i].y;
  }
  gsk::rdft<N>(a);
  double err = 0, nrm = 0;
  for (int k = 0; k < N; ++k) {
    double sr = 0, si = 0;
    for (int n = 0; n < N; ++n) {
      const double ang = -2.0 * M_PI * static_cast<double>((static_cast<long>(n) * k) % N) / N;
      sr += xr[n] * std::cos(ang) - xi[n] * std::sin(ang);
      si += xr[n] * std::sin(ang) + xi[n] * std::cos(ang);
    }
    err += (sr - a[k].x) * (sr - a[k].x) + (si - a[k].y) * (si - a[k].y);
    nrm += sr * sr + si * si;
  }
  return std::sqrt(err / nrm);
}

int main() {
  std::printf("3 %.3e\n", check<3>());
  std::printf("5 %.3e\n", check<5>());
  std::printf("6 %.3e\n", check<6>());
  std::printf("9 %.3e\n", check<9>());
  std::printf("10 %.3e\n", check<10>());
  std::printf("12 %.3e\n", check<12>());
  std::printf("15 %.3e\n", check<15>());
  std::printf("20 %.3e\n", check<20>());
  std::printf("24 %.3e\n", check<24>());
  std::printf("25 %.3e\n", check<25>());
  std::printf("27 %.3e\n", check<27>());
  std::printf("30 %.3e\n", check<30>());
  std::printf("32 %.3e\n", check<32>());
  double worst = 0;
  for (int n = 1; n <= 64; ++n)
    for (int m = -n; m < 2 * n; ++m) {
      const gsk::CosSin w = gsk::unit_cs(m, n);
      worst = std::fmax(worst, std::fmax(std::fabs(w.c - std::cos(2 * M_PI * m / n)), std::fabs(w.s - std::sin(2 * M_PI * m / n))));
    }
  std::printf("cs %.3e\n", worst);
  return 0;
}
