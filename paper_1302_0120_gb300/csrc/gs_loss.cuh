// gs_loss.cuh -- intensity loss and its adjoint (gradient) in one persistent
// launch, for square grids.
//
// The differentiable form of the same inverse problem (fit |F u|^2 to the
// target intensity over phase-only u, Sec. II):
//   L(phi) = sum_k (|y_k|^2 / N - I_k)^2,   y = F x,  x = exp(i phi)
//   dL/dphi_j = 4 Im(conj(x_j) z_j),        z = F^{-1}(r * y),  r = |y|^2/N - I
// with F the unnormalised 2D DFT and F^{-1} its normalised inverse (from
// dy_k/dphi_j = F_kj i x_j and the symmetry of F). Three passes:
//   rows     x = exp(i phi), B = DFT_x(x)                       (as A1)
//   columns  y = DFT_y(B); r; loss partial; B = IDFT_y(r * y)   (adjoint, swapped)
//   rows     N z = IDFT_x(B); grad = 4 Im(conj(x) z)            (adjoint)
// The target is staged like the amplitude of the iteration kernel
// (transposed [nx][ny], read per column block). FP64 only for the loss sum.
#pragma once

#include "gs_iterate.cuh"

namespace gsk {

// Grid barrier for the loss kernel (same protocol as grid_sync).
static __device__ bool loss_sync(const LossParams& p, unsigned& target, Shared& sh) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(p.bar, 1u);
    unsigned spins = 0;
    unsigned long long t0 = 0;
    while (static_cast<int>(ld_acquire_gpu(p.bar) - target) < 0) {
      ++spins;
      if ((spins & 255u) == 0) {
        const unsigned long long now = global_ns();
        if (t0 == 0) t0 = now;
        if (now - t0 > kBarrierTimeoutNs || spins > kMaxSpins) {
          ok = 0;
          atomicCAS(p.status, 0, GS_ETIMEOUT);
          atomicExch(p.abort_flag, 1);
          break;
        }
      }
    }
    __threadfence();
    if (ok && *reinterpret_cast<volatile int*>(p.abort_flag) != 0) ok = 0;
    sh.flag = ok;
  }
  __syncthreads();
  return sh.flag != 0;
}

template <int LN>
__global__ void __launch_bounds__(kThreads, 1) gs_loss_kernel(const LossParams p) {
  using G = GroupT<LN>;
  using L = FieldLayout<LN, LN>;
  constexpr int N = G::N;
  constexpr int T = G::T;
  constexpr int LOGT = LN - 5;
  constexpr int NG = kThreads / T;
  constexpr int W = L::W;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shared sh;
  const int b = blockIdx.x;
  const int gidx = threadIdx.x >> LOGT;
  G grp;
  grp.t = threadIdx.x & (T - 1);
  grp.bar_id = 1 + gidx;
  grp.sm = reinterpret_cast<float2*>(smem) + gidx * G::SMEM;
  grp.tw = p.tw;
  const int t = grp.t;
  StageTw<LN> stw;
  stw.load(p.tw, t);
  float* its = reinterpret_cast<float*>(smem + kAmpSmemOffset);
  float2* blk = reinterpret_cast<float2*>(smem + kBlockSmemOffset);
  unsigned target = 0;
  unsigned mphase = 0;
  if (threadIdx.x == 0) {
    mbar_init(&sh.mbar, 1);
    fence_barrier_init();
    sh.pending = 0;
  }
  __syncthreads();

  // Target: validate this block's rows, and stage its columns transposed.
  {
    const int r0 = split(b, gridDim.x, N);
    const int r1 = split(b + 1, gridDim.x, N);
    bool bad = false;
    for (int e = threadIdx.x; e < (r1 - r0) * N; e += kThreads) {
      const float x = p.I[static_cast<size_t>(r0) * N + e];
      bad |= !(fabsf(x) <= FLT_MAX);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) p.partials[b] = __longlong_as_double(0x7ff8000000000000ll);
    else if (threadIdx.x == 0) p.partials[b] = 0.0;
    // transpose this block's column blocks through shared memory (coalesced
    // on both sides): IT[c][y] = I[y][c]
    const int lo = split(b, gridDim.x, L::NBLK);
    const int hi = split(b + 1, gridDim.x, L::NBLK);
    float* tb = reinterpret_cast<float*>(blk);  // [N][W + 1]
    for (int cb = lo; cb < hi; ++cb) {
      __syncthreads();
      for (int e = threadIdx.x; e < N * W; e += kThreads) {
        const int k = e & (W - 1);
        const int y = e >> L::LW;
        tb[y * (W + 1) + k] = p.I[static_cast<size_t>(y) * N + cb * W + k];
      }
      __syncthreads();
      for (int e = threadIdx.x; e < N * W; e += kThreads) {
        const int k = e >> LN;
        const int y = e & (N - 1);
        p.IT[static_cast<size_t>(cb * W + k) * N + y] = tb[y * (W + 1) + k];
      }
    }
  }

  // Pass 1 (rows): x = exp(i phi), B = DFT_x(x).
  {
    const int lo = split(b, gridDim.x, N);
    const int hi = split(b + 1, gridDim.x, N);
    for (int base = lo; base < hi; base += NG) {
      const int idx = base + gidx;
      const bool valid = idx < hi;
      const int ridx = valid ? idx : base;
      float2 v[32];
      const float* ph = p.phi + static_cast<size_t>(ridx) * N + t;
      float2* su = grp.sm + t;
#pragma unroll 1
      for (int i = 0; i < 32; ++i) {
        float s, c;
        sincosf(ph[T * i], &s, &c);
        su[T * i] = make_float2(c, s);
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = su[T * i];
      grp.sync();
      group_fft<LN>(v, grp, stw);
      if (valid) {
#pragma unroll
        for (int i = 0; i < 32; ++i) p.B[L::off(idx, t + T * i)] = v[i];
      }
    }
  }
  if (!loss_sync(p, target, sh)) return;
  {
    double tot = 0.0;
    for (int c = 0; c < static_cast<int>(gridDim.x); ++c) tot += p.partials[c];
    if (!(tot == 0.0)) {  // a non-finite target
      if (b == 0 && threadIdx.x == 0) {
        atomicCAS(p.status, 0, GS_ENUMERIC);
        p.loss[0] = __longlong_as_double(0x7ff8000000000000ll);
      }
      return;
    }
  }

  // Pass 2 (columns): y = DFT_y(B) = F x; r = |y|^2/N - I; loss partial;
  // B = swap(IDFT_y(r y)) for the adjoint.
  const bool want_grad = p.grad != nullptr;
  double acc = 0.0;
  {
    const int lo = split(b, gridDim.x, L::NBLK);
    const int hi = split(b + 1, gridDim.x, L::NBLK);
    const bool gact = gidx < W;
    const bool wact = ((threadIdx.x & ~31) >> LOGT) < W;
    const int gq = gact ? gidx : 0;
    for (int cb = lo; cb < hi; ++cb) {
      __syncthreads();
      if (threadIdx.x == 0) {
        bulk_wait_read_all();
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&sh.mbar, L::BLOCK * 12u);
        bulk_g2s(blk, p.B + static_cast<size_t>(cb) * L::BLOCK, L::BLOCK * 8u, &sh.mbar);
        bulk_g2s(its, p.IT + static_cast<size_t>(cb) * L::BLOCK, L::BLOCK * 4u, &sh.mbar);
        sh.pending = 1;
        sh.pending_phase = mphase;
      }
      const bool landed = mbar_wait_bounded(&sh.mbar, mphase);
      mphase ^= 1u;
      if (!landed) {
        atomicCAS(p.status, 0, GS_ETIMEOUT);
        atomicExch(p.abort_flag, 1);
      } else if (threadIdx.x == 0) {
        sh.pending = 0;
      }
      if (wact) {
        float2 v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = blk[L::boff(t + T * i, gq)];
        group_fft<LN>(v, grp, stw);
        const float* icol = its + gq * N + t;
        float part = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float2 y = v[i];
          const float r = (y.x * y.x + y.y * y.y) * p.inv_n - icol[T * i];
          part = fmaf(r, r, part);
          v[i] = make_float2(r * y.y, r * y.x);  // swapped: the next forward DFT acts as the inverse
        }
        if (gact) acc += static_cast<double>(part);
        if (want_grad) {
          group_fft<LN>(v, grp, stw);
          if (gact) {
#pragma unroll
            for (int i = 0; i < 32; ++i) blk[L::boff(t + T * i, gidx)] = v[i];
          }
        }
      }
      if (want_grad) {
        __syncthreads();
        if (threadIdx.x == 0) {
          fence_proxy_async_smem();
          bulk_s2g(p.B + static_cast<size_t>(cb) * L::BLOCK, blk, L::BLOCK * 8u);
          bulk_commit();
        }
      }
    }
    if (want_grad && threadIdx.x == 0) bulk_wait_all();
  }
  {
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) p.partials[gridDim.x + b] = tot;
  }
  if (!loss_sync(p, target, sh)) {
    if (threadIdx.x == 0 && sh.pending) mbar_wait_bounded(&sh.mbar, sh.pending_phase);
    return;
  }
  if (b == 0 && threadIdx.x < 32) {
    double s = 0.0;
    for (int c = threadIdx.x; c < static_cast<int>(gridDim.x); c += 32) s += p.partials[gridDim.x + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) p.loss[0] = s;
  }
  if (!want_grad) return;

  // Pass 3 (rows): N z = IDFT_x(B), grad = 4 Im(conj(x) z) with x = exp(i phi).
  {
    const int lo = split(b, gridDim.x, N);
    const int hi = split(b + 1, gridDim.x, N);
    const float scale = 4.f * p.inv_n;
    for (int base = lo; base < hi; base += NG) {
      const int idx = base + gidx;
      const bool valid = idx < hi;
      const int ridx = valid ? idx : base;
      float2 v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = p.B[L::off(ridx, t + T * i)];
      group_fft<LN>(v, grp, stw);  // = swap(N z)
      // Im(conj(x) z) = x.re z.im - x.im z.re, with z = (v.y, v.x) / N
      float2* su = grp.sm + t;
#pragma unroll
      for (int i = 0; i < 32; ++i) su[T * i] = v[i];
      if (valid) {
        const float* ph = p.phi + static_cast<size_t>(idx) * N + t;
        float* gr = p.grad + static_cast<size_t>(idx) * N + t;
#pragma unroll 1
        for (int i = 0; i < 32; ++i) {
          float s, c;
          sincosf(ph[T * i], &s, &c);
          const float2 w = su[T * i];
          gr[T * i] = scale * (c * w.x - s * w.y);
        }
      }
      grp.sync();
    }
  }
}

}  // namespace gsk
