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
// (transposed [nx][ny], read per column block). FP64 only for the sums.
// With the Adam update fused into the third pass, one launch can run many
// optimiser steps: the third pass of a step, which owns the same rows as the
// first, also forms the next step's x = exp(i phi) and B = DFT_x(x), so every
// step after the first is a column pass and a row pass.
// With a laser amplitude p on the SLM the field is x = p exp(i phi); the
// gradient formula is unchanged (dy_k/dphi_j = F_kj i x_j still holds).
//
// The same column pass can also evaluate the physical error of Eq.
// (phys-error) for u = x (Sec. II): with It = I / max I and the reconstructed
// intensity Ir = |F_u u|^2 (sum I / sum p^2) / max I,
//   E_l = sum_{I > 0} (t_d |It - Ir| / (t_l It) - t_d) Theta(|It - Ir|/It - t_l)
//   E_d = sum_{I = 0} (Ir - t_d) Theta(Ir - t_d),   t_l = 0.1, t_d = 3e-4.
#pragma once

#include "gs_iterate.cuh"

namespace gsk {

constexpr float kTolLit = 0.1f;    // t_l, Sec. II
constexpr float kTolDark = 3e-4f;  // t_d, Sec. II

// partial-sum rows of the loss kernel (each [grid]); row kRowStaged holds the
// reduced target statistics of a prepared target (flag, sum I, max I).
enum LossRow { kRowFlag = 0, kRowSumI = 1, kRowMaxI = 2, kRowLoss = 3, kRowEl = 4, kRowEd = 5, kRowStaged = 6 };

// Record a failure: the first one also adds the abort bit to the barrier
// counter, which releases every waiting block (as fail() in gs_common.cuh).
static __device__ void loss_fail(const LossParams& p, int code) {
  atomicCAS(p.status, 0, code);
  if (atomicExch(p.abort_flag, 1) == 0) atomicAdd(p.bar, kAbortBit);
}

// Grid barrier for the loss kernel (same protocol as grid_sync).
static __device__ bool loss_sync(const LossParams& p, unsigned& target, Shared& sh) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    int ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p.bar) : "memory");
    unsigned spins = 0;
    unsigned long long t0 = 0;
    unsigned v;
    while (static_cast<int>((v = ld_acquire_gpu(p.bar)) - target) < 0) {
      ++spins;
      if ((spins & 255u) == 0) {
        const unsigned long long now = global_ns();
        if (t0 == 0) t0 = now;
        if (now - t0 > kBarrierTimeoutNs || spins > kMaxSpins) {
          ok = 0;
          loss_fail(p, GS_ETIMEOUT);
          break;
        }
      }
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (ok && (v & kAbortBit) != 0) ok = 0;  // a block failed in this launch
    sh.flag = ok;
  }
  __syncthreads();
  return sh.flag != 0;
}

// MODE (LossMode, gs_internal.h) kLossFused: validate and stage the target,
// then the three passes (one call does everything). kLossPrepare: validate
// and stage the target only, and reduce its statistics into row kRowStaged.
// kLossStep: the three passes on the staged target (the target of the last
// kLossPrepare launch); with the Adam update, p.steps optimiser steps.

template <int LN, int MODE>
__global__ void __launch_bounds__(kThreads, 1) gs_loss_kernel(const LossParams p) {
  using G = GroupT<LN>;
  using L = FieldLayout<LN, LN, false>;
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
  if constexpr (MODE != kLossStep) {
    const int r0 = split(b, gridDim.x, N);
    const int r1 = split(b + 1, gridDim.x, N);
    bool bad = false;
    double sum_i = 0.0;
    float max_i = 0.f;
    const float* Ib = p.I + static_cast<size_t>(r0) * N;
    const int cnt = (r1 - r0) * N;
    for (int e0 = threadIdx.x; e0 < cnt; e0 += 8 * kThreads) {
      float xs[8];  // eight loads in flight before they are used
#pragma unroll
      for (int u = 0; u < 8; ++u) xs[u] = (e0 + u * kThreads < cnt) ? Ib[e0 + u * kThreads] : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        bad |= !(fabsf(xs[u]) <= FLT_MAX);
        sum_i += static_cast<double>(xs[u]);
        max_i = fmaxf(max_i, xs[u]);
      }
    }
    const int any_bad = __syncthreads_or(bad);
    const double bsum = block_sum(sum_i, sh);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) max_i = fmaxf(max_i, __shfl_xor_sync(0xffffffffu, max_i, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = static_cast<double>(max_i);
    __syncthreads();
    if (threadIdx.x == 0) {
      double bmax = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) bmax = fmax(bmax, sh.red[w]);
      const int G = gridDim.x;
      p.partials[kRowFlag * G + b] = any_bad ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
      p.partials[kRowSumI * G + b] = bsum;
      p.partials[kRowMaxI * G + b] = bmax;
    }
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
        cp_async4(tb + y * (W + 1) + k, p.I + static_cast<size_t>(y) * N + cb * W + k);
      }
      cp_async_wait_all();
      __syncthreads();
      for (int e = threadIdx.x; e < N * W; e += kThreads) {
        const int k = e >> LN;
        const int y = e & (N - 1);
        p.IT[static_cast<size_t>(cb * W + k) * N + y] = tb[y * (W + 1) + k];
      }
    }
  }
  if constexpr (MODE == kLossPrepare) {
    // the staged target's statistics, reduced once (FP64, fixed order)
    if (!loss_sync(p, target, sh)) return;
    if (b == 0 && threadIdx.x == 0) {
      const int G = gridDim.x;
      double flag = 0.0, sum_i = 0.0, max_i = 0.0;
      for (int c = 0; c < G; ++c) {
        flag += p.partials[kRowFlag * G + c];
        sum_i += p.partials[kRowSumI * G + c];
        max_i = fmax(max_i, p.partials[kRowMaxI * G + c]);
      }
      double* st = p.partials + kRowStaged * kMaxGrid;  // a fixed place: the step may use another grid
      st[0] = flag;
      st[1] = sum_i;
      st[2] = max_i;
      if (!(flag == 0.0)) atomicCAS(p.status, 0, GS_ENUMERIC);
    }
    return;
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
      const float* pp = p.p_slm ? p.p_slm + static_cast<size_t>(ridx) * N + t : nullptr;
      float2* su = grp.sm + t;
      // phi (and p) by cp.async, all loads in flight, then a rolled loop
#pragma unroll
      for (int i = 0; i < 32; ++i) cp_async4(&su[T * i].x, ph + T * i);
      if (pp) {
#pragma unroll
        for (int i = 0; i < 32; ++i) cp_async4(&su[T * i].y, pp + T * i);
      }
      cp_async_wait_all();
      // four copies of sincosf: independent work for the scheduler, while
      // the code stays small (instruction fetch is this kernel's top stall)
#pragma unroll 4
      for (int i = 0; i < 32; ++i) {
        float s, c;
        const float2 fa = su[T * i];
        sincosf(fa.x, &s, &c);
        const float a = pp ? fa.y : 1.f;
        su[T * i] = make_float2(a * c, a * s);
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
  // Scale of the reconstructed intensity for the physical error:
  // Ir = |y|^2/N * (sum I / sum p^2) / max I, It = I / max I.
  float ir_scale = 0.f, it_scale = 0.f;
  {
    double tot = 0.0, sum_i = 0.0, max_i = 0.0;
    const int G = gridDim.x;
    if constexpr (MODE == kLossStep) {
      const double* st = p.partials + kRowStaged * kMaxGrid;  // written by the prepare launch
      tot = st[0];
      sum_i = st[1];
      max_i = st[2];
    } else {
      for (int c = 0; c < G; ++c) {
        tot += p.partials[kRowFlag * G + c];
        sum_i += p.partials[kRowSumI * G + c];
        max_i = fmax(max_i, p.partials[kRowMaxI * G + c]);
      }
    }
    const double ep = p.p_slm ? *p.energy : static_cast<double>(N) * N;
    if (max_i > 0.0 && ep > 0.0) {
      ir_scale = static_cast<float>((sum_i / ep) / max_i * p.inv_n);
      it_scale = static_cast<float>(1.0 / max_i);
    }
    if (!(tot == 0.0) || (p.p_slm && !(ep > 0.0 && ep <= DBL_MAX))) {  // a non-finite target or a bad p
      if (b == 0 && threadIdx.x == 0) {
        atomicCAS(p.status, 0, GS_ENUMERIC);
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        for (int k = 0; k < (p.m != nullptr ? p.steps : 1); ++k) p.loss[k] = nan;
        if (p.phys) p.phys[0] = p.phys[1] = nan;
      }
      return;
    }
  }

  const bool adam = p.m != nullptr;  // the Adam update in place of the gradient output
  const bool want_grad = p.grad != nullptr || adam;  // the adjoint passes
  const bool want_phys = p.phys != nullptr;
  // Adam steps of this launch; every block reads the step count before the
  // last block to finish advances it
  const int steps = adam ? p.steps : 1;
  const int t_done = adam ? p.state[0] : 0;
  for (int k = 0; k < steps; ++k) {
    // Pass 2 (columns): y = DFT_y(B) = F x; r = |y|^2/N - I; loss partial;
    // B = swap(IDFT_y(r y)) for the adjoint.
    float acc = 0.f, acc_l = 0.f, acc_d = 0.f;  // this thread's lines, FP32
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
          loss_fail(p, GS_ETIMEOUT);
        } else if (threadIdx.x == 0) {
          sh.pending = 0;
        }
        if (wact) {
          float2 v[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = blk[L::boff(t + T * i, gq)];
          group_fft<LN>(v, grp, stw);
          const float* icol = its + gq * N + t;
          float* sa2 = reinterpret_cast<float*>(grp.sm) + t;  // |y|^2 for the physical error
          float part = 0.f;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float2 y = v[i];
            const float a2 = y.x * y.x + y.y * y.y;
            const float r = a2 * p.inv_n - icol[T * i];
            part = fmaf(r, r, part);
            if (want_phys) sa2[T * i] = a2;
            v[i] = make_float2(r * y.y, r * y.x);  // swapped: the next forward DFT acts as the inverse
          }
          if (gact) acc += part;
          if (want_phys) {  // Eq. (phys-error), once per call: a rolled loop
            float el = 0.f, ed = 0.f;
#pragma unroll 1
            for (int i = 0; i < 32; ++i) {
              const float ir = sa2[T * i] * ir_scale;  // reconstructed intensity
              const float iv = icol[T * i];
              if (iv > 0.f) {
                const float it = iv * it_scale;
                const float rel = fabsf(it - ir) / it;
                if (rel - kTolLit > 0.f) el += kTolDark * rel / kTolLit - kTolDark;
              } else if (ir - kTolDark > 0.f) {
                ed += ir - kTolDark;
              }
            }
            if (gact) {
              acc_l += el;
              acc_d += ed;
            }
            grp.sync();
          }
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
      const int G = gridDim.x;
      // FP32 within the block, FP64 across blocks (below)
      const double tot = block_sum_f(acc, sh);
      if (threadIdx.x == 0) p.partials[kRowLoss * G + b] = tot;
      if (want_phys) {
        const double tl = block_sum_f(acc_l, sh);
        if (threadIdx.x == 0) p.partials[kRowEl * G + b] = tl;
        const double td = block_sum_f(acc_d, sh);
        if (threadIdx.x == 0) p.partials[kRowEd * G + b] = td;
      }
    }
    if (!loss_sync(p, target, sh)) {
      if (threadIdx.x == 0 && sh.pending) mbar_wait_bounded(&sh.mbar, sh.pending_phase);
      return;
    }
    // Block 0 reads the partials here and reaches the barrier that lets the
    // other blocks write the next step's partials only after that.
    if (b == 0 && threadIdx.x < 32) {
      const int G = gridDim.x;
      for (int row = kRowLoss; row <= (want_phys ? kRowEd : kRowLoss); ++row) {
        double s = 0.0;
        for (int c = threadIdx.x; c < G; c += 32) s += p.partials[row * G + c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) {
          if (row == kRowLoss) p.loss[k] = s;
          else p.phys[row - kRowEl] = s;
        }
      }
    }
    if (!want_grad) return;

    // Pass 3 (rows): N z = IDFT_x(B), grad = 4 Im(conj(x) z) with x = exp(i phi);
    // with the fused update, the Adam step of gs_adam_step on every element
    // instead of its gradient output (the phase of a row is read into shared
    // memory before the thread that owns each element updates it). When
    // another step follows, the same pass also does its pass 1 for the rows it
    // owns (the rows are split over the blocks as in pass 1): exp(i phi) of
    // the updated phase, straight from the update, then B = DFT_x through a
    // second turn of the transform loop.
    const bool fuse = k + 1 < steps;
    int adam_t = 0;
    float adam_step = 0.f, adam_rb2 = 0.f;
    if (adam) {
      adam_t = t_done + 1 + k;
      const float b1 = 1.f - powf(p.beta1, static_cast<float>(adam_t));
      const float b2 = 1.f - powf(p.beta2, static_cast<float>(adam_t));
      adam_step = p.lr / b1;
      adam_rb2 = 1.f / sqrtf(b2);
    }
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
        // phi (and p) of this row by cp.async into the field staging buffer
        // (free in this pass), in flight behind the transform
        float* sph = reinterpret_cast<float*>(blk) + threadIdx.x;
        float* spp = sph + 32 * kThreads;
        // the fused update with p = 1: the row's moments too, into the laser
        // amplitude's buffer and the staged target's (free in this pass)
        float* const smm = (adam && !p.p_slm) ? spp : nullptr;
        float* const smv = (adam && !p.p_slm) ? its + threadIdx.x : nullptr;
        {
          const size_t r0 = static_cast<size_t>(ridx) * N + t;
          const float* ph = p.phi + r0;
#pragma unroll
          for (int i = 0; i < 32; ++i) cp_async4(sph + kThreads * i, ph + T * i);
          if (p.p_slm) {
            const float* pp = p.p_slm + r0;
#pragma unroll
            for (int i = 0; i < 32; ++i) cp_async4(spp + kThreads * i, pp + T * i);
          }
          if (smm != nullptr) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              cp_async4(smm + kThreads * i, p.m + r0 + T * i);
              cp_async4(smv + kThreads * i, p.v + r0 + T * i);
            }
          }
        }
        // one copy of the transform for both turns (instruction fetch is this
        // kernel's top stall)
#pragma unroll 1
        for (int h = 0; h < (fuse ? 2 : 1); ++h) {
          group_fft<LN>(v, grp, stw);  // h = 0: swap(N z); h = 1: the next step's row DFT
          if (h == 1) {
            if (valid) {
#pragma unroll
              for (int i = 0; i < 32; ++i) p.B[L::off(idx, t + T * i)] = v[i];
            }
            break;
          }
          // Im(conj(x) z) = x.re z.im - x.im z.re, with z = (v.y, v.x) / N
          float2* su = grp.sm + t;
#pragma unroll
          for (int i = 0; i < 32; ++i) su[T * i] = v[i];
          cp_async_wait_all();
          if (valid && !adam) {
            float* gr = p.grad + static_cast<size_t>(idx) * N + t;
#pragma unroll 4
            for (int i = 0; i < 32; ++i) {
              float s, c;
              sincosf(sph[kThreads * i], &s, &c);
              const float a = p.p_slm ? spp[kThreads * i] : 1.f;  // x = p exp(i phi)
              const float2 w = su[T * i];
              gr[T * i] = scale * a * (c * w.x - s * w.y);
            }
          } else if (valid) {
            const size_t e0 = static_cast<size_t>(idx) * N + t;
#pragma unroll 4
            for (int i = 0; i < 32; ++i) {
              float s, c;
              sincosf(sph[kThreads * i], &s, &c);
              const float a = p.p_slm ? spp[kThreads * i] : 1.f;
              const float2 w = su[T * i];
              const float g = scale * a * (c * w.x - s * w.y);
              const size_t e = e0 + T * i;
              const float m0 = smm ? smm[kThreads * i] : p.m[e];
              const float v0 = smv ? smv[kThreads * i] : p.v[e];
              const float mi = fmaf(p.beta1, m0, (1.f - p.beta1) * g);
              const float vi = fmaf(p.beta2, v0, (1.f - p.beta2) * g * g);
              p.m[e] = mi;
              p.v[e] = vi;
              const float ph = sph[kThreads * i] - adam_step * mi / (sqrtf(vi) * adam_rb2 + p.eps);
              p.phase[e] = ph;
              if (fuse) {  // x = p exp(i phi) of the next step, in place of w
                sincosf(ph, &s, &c);
                su[T * i] = make_float2(a * c, a * s);
              }
            }
          }
          if (fuse) {  // a group with no row of its own transforms what it holds and stores nothing
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = su[T * i];
            grp.sync();
          }
        }
        grp.sync();
      }
    }
    if (fuse && !loss_sync(p, target, sh)) return;
  }  // steps
  if (adam) {  // the last block to finish advances the step count (every block has read it)
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(p.state + 1, 1) == static_cast<int>(gridDim.x) - 1) {
        p.state[0] = t_done + steps;
        p.state[1] = 0;
      }
    }
  }
}

}  // namespace gsk
