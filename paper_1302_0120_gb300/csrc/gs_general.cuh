// gs_general.cuh -- passes of the iteration kernel for grids whose sides are
// not powers of two (any 5-smooth side 2^a 3^b 5^c in [32, 1536]), such as
// the 800 x 600 SLM of Sec. V.
//
// The pass structure, projections and FP64 gap sums are those of the
// power-of-two kernel (gs_iterate.cuh); what differs is the transform and the
// data movement:
//   * The field B is stored row-major [ny][nx]; m transposed [nx][ny].
//   * A row or column is transformed by a team of two warps (64 threads,
//     four teams per block), which halves each transform's chain of
//     dependent stage loops; teams synchronise on their own named barrier.
//   * A row pass gives each team one row: the row is read coalesced into the
//     team's shared-memory buffer, transformed, projected and transformed
//     again there, and written back coalesced.
//   * A column pass moves 4 adjacent columns at a time: the block reads the
//     [ny][4] tile in 32-byte row segments into four per-team column buffers,
//     each team transforms, projects and transforms its column, and the block
//     writes the tile back the same way.
//   * A length-n transform is a Stockham auto-sort FFT with radices 3 and 5
//     first, then 8, 4 and 2 (gen_fft), each stage read from one of the warp's
//     two buffers and written to the other. The
//     twiddles of the stage with sub-transform length ns and radix R sit at
//     entries ns - 1 + (m - 1) ns + r (W_{ns R}^{r m}), so that consecutive
//     butterflies read consecutive entries; the tables are rounded once from
//     double on the host and copied to shared memory per launch.
//   * Rows and column tiles arrive by cp.async, every copy of a thread in
//     flight at once.
#pragma once

#include "gs_common.cuh"
#include "gs_fft.cuh"
#include "gs_tma.cuh"

namespace gsk {

// Radix of stage code c (3 bits per stage in Params::planx / plany).
__host__ __device__ constexpr int radix_of_code(unsigned c) {
  return c == 0 ? 2 : c == 1 ? 3 : c == 2 ? 4 : c == 3 ? 5 : 8;
}

// 3-point DFT, exp(-2 pi i jk/3): with t = a1 + a2 and d = (sqrt3/2)(a1 - a2),
// y1,2 = a0 - t/2 -/+ i d.
__host__ __device__ __forceinline__ void dft3(float2 (&a)[3]) {
  constexpr float h = 0.8660254037844386f;  // sqrt(3)/2
  const float2 t = cadd(a[1], a[2]);
  const float2 d = make_float2(h * (a[1].x - a[2].x), h * (a[1].y - a[2].y));
  const float2 c = make_float2(fmaf(-0.5f, t.x, a[0].x), fmaf(-0.5f, t.y, a[0].y));
  a[0] = cadd(a[0], t);
  a[1] = make_float2(c.x + d.y, c.y - d.x);
  a[2] = make_float2(c.x - d.y, c.y + d.x);
}

// 5-point DFT, exp(-2 pi i jk/5), from the symmetric and antisymmetric pairs
// b1 = a1 + a4, b2 = a2 + a3, d1 = a1 - a4, d2 = a2 - a3:
//   y1,4 = a0 + c1 b1 + c2 b2 -/+ i (s1 d1 + s2 d2)
//   y2,3 = a0 + c2 b1 + c1 b2 -/+ i (s2 d1 - s1 d2)
// with ck = cos(2 pi k/5), sk = sin(2 pi k/5).
__host__ __device__ __forceinline__ void dft5(float2 (&a)[5]) {
  constexpr float c1 = 0.30901699437494745f, c2 = -0.8090169943749475f;
  constexpr float s1 = 0.9510565162951535f, s2 = 0.5877852522924731f;
  const float2 b1 = cadd(a[1], a[4]), b2 = cadd(a[2], a[3]);
  const float2 d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
  const float2 e1 = make_float2(fmaf(c1, b1.x, fmaf(c2, b2.x, a[0].x)), fmaf(c1, b1.y, fmaf(c2, b2.y, a[0].y)));
  const float2 e2 = make_float2(fmaf(c2, b1.x, fmaf(c1, b2.x, a[0].x)), fmaf(c2, b1.y, fmaf(c1, b2.y, a[0].y)));
  const float2 f1 = make_float2(fmaf(s1, d1.x, s2 * d2.x), fmaf(s1, d1.y, s2 * d2.y));
  const float2 f2 = make_float2(fmaf(s2, d1.x, -s1 * d2.x), fmaf(s2, d1.y, -s1 * d2.y));
  a[0] = cadd(a[0], cadd(b1, b2));
  // e - i f = (e.x + f.y, e.y - f.x)
  a[1] = make_float2(e1.x + f1.y, e1.y - f1.x);
  a[4] = make_float2(e1.x - f1.y, e1.y + f1.x);
  a[2] = make_float2(e2.x + f2.y, e2.y - f2.x);
  a[3] = make_float2(e2.x - f2.y, e2.y + f2.x);
}

template <int R>
__host__ __device__ __forceinline__ void small_dft(float2 (&a)[R]) {
  if constexpr (R == 3) dft3(a);
  else if constexpr (R == 5) dft5(a);
  else dft<R>(a);
}

// Barrier of team `team` (its two warps), named barrier 1 + team.
__device__ __forceinline__ void team_sync(int team) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "n"(kGenTeam) : "memory");
}

// One Stockham stage of radix R on a length-n transform whose first stages
// formed sub-transforms of length ns: butterfly j = q ns + r reads
// src[j + m n/R], multiplies by W_{ns R}^{r m} (stage table tw), transforms
// over m and writes dst[q ns R + r + k ns]. Thread t of the team takes
// butterflies t, t + 64, ...
template <int R>
__device__ __forceinline__ void gen_stage(const float2* __restrict__ src, float2* __restrict__ dst, int n, int ns,
                                          const float2* __restrict__ tw) {
  constexpr int U = 1;
  const int nb = n / R;
  const int tt = threadIdx.x % kGenTeam;
  const int qinc = kGenTeam / ns, rinc = kGenTeam % ns;
  int q = tt / ns, r = tt % ns;
  const float2* const tws = tw + (ns - 1);
  for (int j0 = tt; j0 < nb; j0 += kGenTeam * U) {
    float2 a[U][R];
    int base[U], rr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + kGenTeam * u;
      rr[u] = r;
      base[u] = q * ns * R + r;
      if (j < nb) {
#pragma unroll
        for (int m = 0; m < R; ++m) a[u][m] = src[j + m * nb];
      }
      q += qinc;
      r += rinc;
      if (r >= ns) {
        r -= ns;
        ++q;
      }
    }
    if (ns > 1) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (j0 + kGenTeam * u < nb) {
#pragma unroll
          for (int m = 1; m < R; ++m) a[u][m] = cmul(a[u][m], tws[(m - 1) * ns + rr[u]]);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + kGenTeam * u < nb) {
        small_dft<R>(a[u]);
#pragma unroll
        for (int k = 0; k < R; ++k) dst[base[u] + k * ns] = a[u][k];
      }
  }
}

// Forward unnormalised DFT of the length-n vector in `a` by team `team`,
// using `b` as the second buffer; returns the buffer that holds the result
// (a for an even number of stages, b for an odd one).
__device__ __forceinline__ float2* gen_fft(float2* a, float2* b, int n, unsigned plan, int nst, const float2* tw,
                                           int team) {
  int ns = 1;
#pragma unroll 1
  for (int s = 0; s < nst; ++s) {
    const int R = radix_of_code((plan >> (3 * s)) & 7u);
    switch (R) {
      case 2: gen_stage<2>(a, b, n, ns, tw); break;
      case 3: gen_stage<3>(a, b, n, ns, tw); break;
      case 4: gen_stage<4>(a, b, n, ns, tw); break;
      case 5: gen_stage<5>(a, b, n, ns, tw); break;
      default: gen_stage<8>(a, b, n, ns, tw); break;
    }
    team_sync(team);
    ns *= R;
    float2* t = a;
    a = b;
    b = t;
  }
  return a;
}

// Copy the twiddle tables to shared memory (once per launch).
__device__ __forceinline__ void gen_load_twiddles(const Params& p, unsigned char* smem) {
  float2* t = reinterpret_cast<float2*>(smem);
  for (int e = threadIdx.x; e < p.nx; e += kThreads) t[e] = p.twx[e];
  for (int e = threadIdx.x; e < p.ny; e += kThreads) t[p.nx + e] = p.twy[e];
  __syncthreads();
}

// m = s sqrt(I), transposed ([nx][ny]), for this block's columns.
__device__ __forceinline__ void gen_build_amplitude(const Params& p, int mb, float s) {
  const size_t moff = static_cast<size_t>(mb) * static_cast<size_t>(p.mstride);
  const float* const Im = p.I + moff;
  float* const mTm = p.mT + moff;
  const int lo = split(blockIdx.x, gridDim.x, p.nx);
  const int hi = split(blockIdx.x + 1, gridDim.x, p.nx);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int x = lo + w; x < hi; x += kThreads / 32)
    for (int y = lane; y < p.ny; y += 32)
      mTm[static_cast<size_t>(x) * p.ny + y] = s * sqrtf(Im[static_cast<size_t>(y) * p.nx + x]);
  __syncthreads();
}



// Wrap an angle as the power-of-two kernel does: (-pi, pi].
__device__ __forceinline__ float gen_phase(float2 u) {
  const float a = atan2f(u.y, u.x);
  return (a <= -3.14159274f) ? 3.14159274f : a;
}

// One pass over rows [lo, hi) (kInit, kRow) or 8-column groups [lo, hi)
// (kCol, kResid, kInitM) of mask mb. Returns this thread's FP64 contribution
// to the pass's gap sum.
static __device__ __forceinline__ float run_pass_gen(const Params& p, int mb, int kind, bool last, int lo, int hi,
                                                      unsigned char* smem) {
  const size_t moff = static_cast<size_t>(mb) * static_cast<size_t>(p.mstride);
  float2* const Bm = p.B + moff;
  const float* const mTm = p.mT + moff;
  const int nx = p.nx, ny = p.ny;
  const int nmax = nx > ny ? nx : ny;
  const float2* twx = reinterpret_cast<const float2*>(smem);
  const float2* twy = twx + nx;
  float2* wbase = reinterpret_cast<float2*>(smem) + gen_tw_entries(nx, ny);
  const int tm = threadIdx.x / kGenTeam, tt = threadIdx.x % kGenTeam;
  float2* const A = wbase + tm * gen_team_stride(nmax);
  float2* const Bf = A + nmax + 1;
  const float inv_sqrt_n = p.inv_sqrt_n;
  const bool two = (kind == kCol || (kind == kRow && !(last && !p.final_resid)));
  float acc = 0.f;

  if (kind == kInit || kind == kRow) {
    for (int row = lo + tm; row < hi; row += kGenTeams) {
      float2* src = Bm + static_cast<size_t>(row) * nx;
      const float* pp = p.p_slm ? p.p_slm + static_cast<size_t>(row) * nx : nullptr;
      if (kind == kInit) {
        const float* ph = p.phi_in + moff + static_cast<size_t>(row) * nx;
        float* po = p.phi_out + moff + static_cast<size_t>(row) * nx;
        for (int x0 = tt; x0 < nx; x0 += kGenTeam * 4) {
          float f[4], a[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int x = x0 + kGenTeam * k;
            f[k] = x < nx ? ph[x] : 0.f;
            a[k] = (pp && x < nx) ? pp[x] : 1.f;  // u0 = p exp(i phi0)
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            float s, c;
            sincosf(f[k], &s, &c);
            if (x0 + kGenTeam * k < nx) A[x0 + kGenTeam * k] = make_float2(a[k] * c, a[k] * s);
          }
        }
        if (last) {  // zero iterations
          team_sync(tm);
          for (int x = tt; x < nx; x += kGenTeam) po[x] = gen_phase(A[x]);
        }
      } else {
        for (int x = tt; x < nx; x += kGenTeam) cp_async8(A + x, src + x);
        cp_async_wait_all();
      }
      team_sync(tm);
      float2* res = gen_fft(A, Bf, nx, p.planx, p.nstx, twx, tm);
      if (kind == kRow) {
        // res = swap(IDFT_x(B)) = swap(sqrt(N) P_M u^nu): gap to S, Eq. (e:PS)
        float part = 0.f;
        for (int x0 = tt; x0 < nx; x0 += kGenTeam * 8) {
          float a[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) a[k] = (pp && x0 + kGenTeam * k < nx) ? pp[x0 + kGenTeam * k] : 1.f;
          float2 t8[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) t8[k] = (x0 + kGenTeam * k < nx) ? res[x0 + kGenTeam * k] : make_float2(1.f, 0.f);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int x = x0 + kGenTeam * k;
            if (x < nx) {
              const float2 t = t8[k];
              const float vx = t.y, vy = t.x;
              const float a2 = vx * vx + vy * vy;
              const float rs = rsqrtf(a2);
              const float mag = a2 > 0.f ? a2 * rs : 0.f;
              const float d = mag * inv_sqrt_n - a[k];
              part += d * d;
              const float f = a[k] * rs;
              res[x] = a2 > 0.f ? make_float2(vx * f, vy * f) : make_float2(a[k], 0.f);
            }
          }
        }
        acc += part;
        team_sync(tm);
        if (last) {
          float* po = p.phi_out + moff + static_cast<size_t>(row) * nx;
          for (int x = tt; x < nx; x += kGenTeam) po[x] = gen_phase(res[x]);
        }
        if (two) res = gen_fft(res, res == A ? Bf : A, nx, p.planx, p.nstx, twx, tm);
      }
      if (kind == kInit || two)
        for (int x = tt; x < nx; x += kGenTeam) src[x] = res[x];
      team_sync(tm);
    }
    return acc;
  }

  // Column passes: groups of 4 adjacent columns; team k owns column c0 + k.
  const int stride = gen_team_stride(nmax);
  const bool store = (kind == kCol || kind == kInitM);
  // which of a warp's buffers holds the stored result: A after two transforms,
  // else A or Bf by the parity of the stage count
  const int out_off = (kind == kCol || (p.nsty & 1) == 0) ? 0 : nmax + 1;
  for (int cg = lo; cg < hi; ++cg) {
    const int c0 = cg * kGenTeams;
    const int wc = min(kGenTeams, nx - c0);
    __syncthreads();  // the previous group's tile has been written back
    {
      const int k = threadIdx.x % kGenTeams;  // column of this thread in every round
      if (k < wc) {
        if (kind == kInitM) {
          for (int y = threadIdx.x / kGenTeams; y < ny; y += kThreads / kGenTeams)  // swap((m, 0))
            wbase[k * stride + y] = make_float2(0.f, mTm[static_cast<size_t>(c0 + k) * ny + y]);
        } else {
          for (int y = threadIdx.x / kGenTeams; y < ny; y += kThreads / kGenTeams)
            cp_async8(wbase + k * stride + y, Bm + static_cast<size_t>(y) * nx + c0 + k);
          cp_async_wait_all();
        }
      }
    }
    __syncthreads();
    if (tm < wc) {
      float2* res = gen_fft(A, Bf, ny, p.plany, p.nsty, twy, tm);
      if (kind != kInitM) {
        // res = Y = F u^nu along this column: residual and Eq. (e:Mhat)
        const float* mcol = mTm + static_cast<size_t>(c0 + tm) * ny;
        float part = 0.f;
        for (int y0 = tt; y0 < ny; y0 += kGenTeam * 8) {
          float mv[8];
          float2 yv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) mv[u] = (y0 + kGenTeam * u < ny) ? mcol[y0 + kGenTeam * u] : 0.f;
#pragma unroll
          for (int u = 0; u < 8; ++u) yv[u] = (y0 + kGenTeam * u < ny) ? res[y0 + kGenTeam * u] : make_float2(1.f, 0.f);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int y = y0 + kGenTeam * u;
            if (y < ny) {
              const float m = mv[u];
              const float2 Y = yv[u];
              const float a2 = Y.x * Y.x + Y.y * Y.y;
              const float rs = rsqrtf(a2);
              const float mag = a2 > 0.f ? a2 * rs : 0.f;
              const float d = mag * inv_sqrt_n - m;
              part += d * d;
              if (kind == kCol) {
                const float f = m * rs;
                const float2 Yh = a2 > 0.f ? make_float2(Y.x * f, Y.y * f) : make_float2(m, 0.f);
                res[y] = make_float2(Yh.y, Yh.x);  // swapped: the next forward DFT acts as the inverse
              }
            }
          }
        }
        acc += part;
        team_sync(tm);
        if (kind == kCol) res = gen_fft(res, res == A ? Bf : A, ny, p.plany, p.nsty, twy, tm);
      }
    }
    if (store) {
      __syncthreads();
      for (int e = threadIdx.x; e < ny * kGenTeams; e += kThreads) {
        const int y = e / kGenTeams, k = e % kGenTeams;
        if (k < wc) Bm[static_cast<size_t>(y) * nx + c0 + k] = wbase[k * stride + out_off + y];
      }
    }
  }
  return acc;
}

}  // namespace gsk
