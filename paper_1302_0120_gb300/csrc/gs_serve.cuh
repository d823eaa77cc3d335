// gs_serve.cuh -- a persistent serving kernel: one cooperative launch that
// keeps running Gerchberg-Saxton iterations for the requests a host posts to
// a request table in pinned host memory, admitting new requests between
// iterations (continuous batching without the host between launches).
//
// A server owns S slots; each slot takes requests for square grids n x n of
// any of the sizes 256, 512, 1024 up to the server's largest. The kernel runs
// *ticks*; a tick is one GS iteration of Eq. (e:AP) for every running slot (a
// column pass, a grid barrier, a row pass, a grid barrier), with the per-slot
// work of the other kernels (run_pass, gs_iterate.cuh, dispatched on the
// slot's size; the stage twiddles are loaded per pass, as in the mixed
// launch):
//
//   a slot admitted before tick t:  tick t, column phase: its share of sum I
//                                   (A0); row phase: m = s sqrt(I) (A0) and
//                                   u^0 = exp(i phi_in), B = DFT_x(u^0) (A1)
//   a running slot at iteration nu: column pass (A2, r^nu) and row pass (A3,
//                                   g^nu); the last one writes the phase
//
// so a request of K iterations takes K + 1 ticks, and a request posted while
// others run joins them at the next tick. The target is read, and the phase
// written, directly in the host's pinned buffers; r^nu and g^nu likewise.
//
// Block 0 takes no share of the passes (the other blocks split them); it keeps
// the books instead, beside their passes. It plans each tick at the end of
// the previous one (before the barrier that releases it): it advances every
// slot's state as if the current tick completes, admits the requests posted
// since, and writes the plan into a double buffer that every block reads
// after the barrier. At the start of a tick it finishes the previous one: it
// reduces the row gaps and publishes the requests that completed
// (system-scope fence, then the sequence number in the table); after the
// column barrier it reduces the column gaps. State lives in device memory and advances
// only at planning, so a launch may end between ticks and the next launch
// resumes: a launch leaves when told to stop, after an idle wait, or after
// kServeMaxTicks ticks (which keeps the barrier counter far below its abort
// bit); the host relaunches when requests are outstanding. Every wait is
// bounded: grid barriers (1 s), bulk copies (1 s), the idle wait.
#pragma once

#include "gs_iterate.cuh"

namespace gsk {

constexpr int kServeMaxSlots = 16;
constexpr unsigned kServeMaxTicks = 1u << 20;              // per launch: 2 x 2^20 x 152 arrivals < 2^30
constexpr unsigned long long kServeIdleNs = 20000000ull;  // idle wait before a launch leaves (20 ms)

// One request, written by the host before it bumps req_seq[s].
struct ServeRequest {
  const float* I;       // target intensity [n][n], pinned host memory
  const float* phi_in;  // start phase [n][n], pinned host memory
  float* phi_out;       // final phase [n][n], pinned host memory (may alias phi_in)
  double* r_out;        // r^nu, nu < K (pinned host memory), or null
  double* g_out;        // g^nu, nu < K, or null
  int K;                // iterations, 1 ..
  int n;                // grid n x n: 256, 512 or 1024, at most the server's largest
};

// The request table, in pinned host memory mapped into the device.
struct ServeTable {
  ServeRequest req[kServeMaxSlots];
  unsigned req_seq[kServeMaxSlots];   // host: a new request in slot s when it differs from the served one
  unsigned done_seq[kServeMaxSlots];  // kernel: the last request of slot s completed
  int done_status[kServeMaxSlots];    // kernel: its status (GS_OK, GS_EINVAL, GS_ENUMERIC)
  int stop;                           // host: leave once no request is running
  int running;                        // 1 while a launch serves (host sets it when launching)
  int status;                         // kernel: the device status word when a launch left
};

enum ServeStage { kSlotFree = 0, kSlotAdmitted = 1, kSlotRunning = 2 };
enum ServeColWork { kColNone = 0, kColA0 = 1, kColPass = 2 };
enum ServeRowWork { kRowNone = 0, kRowInit = 1, kRowPass = 2, kRowLast = 3 };

struct ServeSlot {
  int stage;
  int nu;          // next iteration
  int K;
  unsigned seq;    // the request in the slot (or the last one served)
};

struct ServePlan {
  int stop;
  int col[kServeMaxSlots];
  int row[kServeMaxSlots];
  int nu[kServeMaxSlots];
};

// Server state in device memory: slots, per-slot parameters, the plans.
struct ServeState {
  ServeSlot slot[kServeMaxSlots];
  Params p[kServeMaxSlots];
  ServePlan plan[2];
};

struct ServeParams {
  Params base;          // slot arrays (strided by mstride: the largest grid), barrier, status
  const float2* tw[3];  // stage twiddle tables for n = 256, 512, 1024 (null above the largest)
  int max_log;          // log2 of the largest grid
  unsigned max_ticks;   // ticks per launch (kServeMaxTicks; lower only in tests)
  ServeTable* table;    // device address of the mapped request table
  ServeState* st;
  double* part;         // [3][kServeMaxSlots][grid]: A0, column and row partial sums
  int slots;
};

__device__ __forceinline__ unsigned ld_acquire_sys_u32(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* a) {
  int v;
  asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys_u32(unsigned* a, unsigned v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

__device__ __forceinline__ void st_volatile_i32(int* a, int v) {
  asm volatile("st.volatile.global.s32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// Publish the end of request `seq` in slot s: every write of the request
// (made visible to this thread by the grid barrier) before the sequence
// number, at system scope.
__device__ __forceinline__ void serve_publish(ServeTable* tb, int s, unsigned seq, int status) {
  __threadfence_system();
  st_volatile_i32(&tb->done_status[s], status);
  st_release_sys_u32(&tb->done_seq[s], seq);
}

// Admit the request posted in free slot s with sequence number rs (thread 0
// of block 0): its parameters become the slot's Params.
__device__ __forceinline__ void serve_admit(const ServeParams& sp, int s, unsigned rs) {
  ServeState* st = sp.st;
  ServeTable* tb = sp.table;
  const ServeRequest& q = tb->req[s];  // read after the acquire of req_seq
  const float* I = q.I;
  const float* phi_in = q.phi_in;
  float* phi_out = q.phi_out;
  double* r_out = q.r_out;
  double* g_out = q.g_out;
  const int K = q.K;
  const int n = q.n;
  const int ln = (n == 256) ? 8 : (n == 512) ? 9 : (n == 1024) ? 10 : 0;
  st->slot[s].seq = rs;
  if (I == nullptr || phi_in == nullptr || phi_out == nullptr || K < 1 || ln == 0 || ln > sp.max_log) {
    st->slot[s].stage = kSlotFree;
    serve_publish(tb, s, rs, GS_EINVAL);
    return;
  }
  Params p = sp.base;
  const size_t off = static_cast<size_t>(s) * static_cast<size_t>(p.mstride);
  p.B = sp.base.B + off;
  p.mT = sp.base.mT + off;
  p.nx = p.ny = n;
  p.lognx = p.logny = ln;
  p.twx = p.twy = sp.tw[ln - 8];
  p.inv_sqrt_n = 1.f / static_cast<float>(n);
  p.inv_n = 1.0 / (static_cast<double>(n) * n);
  p.I = I;
  p.phi_in = phi_in;
  p.phi_out = phi_out;
  p.r_out = r_out;
  p.g_out = g_out;
  p.mask_flags = sp.base.mask_flags + s;
  p.batch = 1;
  p.iters = K;
  st->p[s] = p;
  st->slot[s].stage = kSlotAdmitted;
  st->slot[s].nu = 0;
  st->slot[s].K = K;
}

// Plan the next tick (warp 0 of block 0, at the end of the current one):
// advance the slots as if the current tick (cur; null at the start of a
// launch) completes, admit requests posted since, decide whether the launch
// leaves. Block 0's sh.bad holds the validity of the slots admitted in cur.
// The lanes read the posted sequence numbers (host memory) in parallel, one
// round trip for all slots; lane 0 does the rest.
__device__ void serve_plan(const ServeParams& sp, const ServePlan* cur, ServePlan* nxt, unsigned ticks,
                           const Shared& sh) {
  ServeState* st = sp.st;
  ServeTable* tb = sp.table;
  const int S = sp.slots;
  const int lane = threadIdx.x & 31;
  if (lane == 0 && cur != nullptr) {
    for (int s = 0; s < S; ++s) {
      ServeSlot& sl = st->slot[s];
      if (cur->col[s] == kColA0) {
        if (sh.bad[s]) {  // nothing of the request was written: publish now
          sl.stage = kSlotFree;
          serve_publish(tb, s, sl.seq, GS_ENUMERIC);
        } else {
          sl.stage = kSlotRunning;
          sl.nu = 0;
        }
      } else if (cur->row[s] == kRowPass) {
        sl.nu += 1;
      } else if (cur->row[s] == kRowLast) {
        sl.stage = kSlotFree;  // published at the start of the next tick
      }
    }
  }
  __syncwarp();
  // admit the requests posted to free slots; true (in every lane) if a slot is busy
  auto admit_posted = [&]() {
    const unsigned mine = lane < S ? ld_acquire_sys_u32(&tb->req_seq[lane]) : 0u;
    int busy = 0;
    for (int s = 0; s < S; ++s) {
      const unsigned rs = __shfl_sync(0xffffffffu, mine, s);
      if (lane == 0) {
        // a new request: acquired again by this lane, which reads its fields
        if (st->slot[s].stage == kSlotFree && rs != st->slot[s].seq)
          serve_admit(sp, s, ld_acquire_sys_u32(&tb->req_seq[s]));
        busy |= (st->slot[s].stage != kSlotFree);
      }
    }
    return __shfl_sync(0xffffffffu, busy, 0) != 0;
  };
  auto stop_asked = [&]() { return __shfl_sync(0xffffffffu, lane == 0 ? ld_volatile_i32(&tb->stop) : 0, 0) != 0; };
  bool any = admit_posted();
  // requests that the current tick completes are published at the start of
  // the next one: never wait idle before that
  bool pending = false;
  if (cur != nullptr)
    for (int s = 0; s < S; ++s) pending = pending || (cur->row[s] == kRowLast);
  int stop = 0;
  if (!any) {
    if (stop_asked() || ticks >= sp.max_ticks) {
      stop = 1;
    } else if (pending) {
      // an empty tick: it publishes, and its own planning waits
    } else {
      // idle: wait (bounded) for a request
      const unsigned long long t0 = global_ns();
      while (!any && global_ns() - t0 < kServeIdleNs) {
        __nanosleep(2000);
        any = admit_posted();
        if (stop_asked()) break;
      }
      if (!any) {
        // leave, unless a request slipped in after the last look: the host
        // reads `running` after posting, so one of the two sees the other
        if (lane == 0) {
          st_volatile_i32(&tb->running, 0);
          __threadfence_system();
        }
        __syncwarp();
        any = admit_posted();
        if (any && lane == 0) st_volatile_i32(&tb->running, 1);
        if (!any) stop = 1;
      }
    }
  } else if (ticks >= sp.max_ticks) {
    stop = 1;  // leave between ticks; the slots resume in the next launch
  }
  if (lane == 0) {
    nxt->stop = stop;
    for (int s = 0; s < S; ++s) {
      const ServeSlot& sl = st->slot[s];
      int c = kColNone, r = kRowNone;
      if (!stop && sl.stage == kSlotAdmitted) {
        c = kColA0;
        r = kRowInit;
      } else if (!stop && sl.stage == kSlotRunning) {
        c = kColPass;
        r = (sl.nu + 1 >= sl.K) ? kRowLast : kRowPass;
      }
      nxt->col[s] = c;
      nxt->row[s] = r;
      nxt->nu[s] = sl.nu;
    }
  }
  __syncwarp();
}

// FP64 sum of the G partials of one slot by warp 0 (the result in every lane).
__device__ __forceinline__ double serve_slot_sum(const double* part, int G) {
  double s = 0.0;
  for (int c = threadIdx.x & 31; c < G; c += 32) s += __ldcg(part + c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// This block's FP64 share of sum I of a slot (its rows); NaN poisons it for
// a negative or non-finite pixel.
__device__ __forceinline__ void serve_a0_partial(const Params& p, double* part, Shared& sh) {
  const int G = gridDim.x, b = blockIdx.x;
  const int r0 = split(b, G, p.ny), r1 = split(b + 1, G, p.ny);
  const float* I = p.I + static_cast<size_t>(r0) * p.nx;
  const int cnt = (r1 - r0) * p.nx;
  double acc = 0.0;
  bool bad = false;
  for (int e = threadIdx.x; e < cnt; e += kThreads) {
    const float x = I[e];
    bad |= !(x >= 0.f && x <= FLT_MAX);
    acc += static_cast<double>(x);
  }
  if (__syncthreads_or(bad)) acc = __longlong_as_double(0x7ff8000000000000ll);
  const double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) part[b] = tot;
}

// One pass of a slot over units [lo, hi) (rows, or column blocks of 8),
// dispatched on the slot's grid.
__device__ __forceinline__ float serve_run_pass(const Params& p, int kind, bool last, int lo, int hi,
                                                unsigned char* smem, Shared& sh, unsigned& mphase) {
  const NoTc tcf{};
  if (p.logny == 8) {
    const StageTw<8> none{};
    return run_pass<8, 8, 8, false>(p, 0, kind, last, lo, hi, smem, sh, mphase, none, tcf);
  }
  if (p.logny == 9) {
    const StageTw<9> none{};
    return run_pass<9, 9, 9, false>(p, 0, kind, last, lo, hi, smem, sh, mphase, none, tcf);
  }
  const StageTw<10> none{};
  return run_pass<10, 10, 10, false>(p, 0, kind, last, lo, hi, smem, sh, mphase, none, tcf);
}

// The persistent serving kernel.
__global__ void __launch_bounds__(kThreads, 1) gs_serve(const ServeParams sp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shared sh;
  __shared__ ServePlan plan;
  __shared__ Params prm[kServeMaxSlots];
  const Params& base = sp.base;
  const int G = gridDim.x, b = blockIdx.x;
  const int S = sp.slots;
  static_assert(FieldLayout<8, 8>::W == 8 && FieldLayout<9, 9>::W == 8 && FieldLayout<10, 10>::W == 8,
                "column blocks of 8 at every size");
  unsigned target = 0, mphase = 0;
  block_setup(sh);
  double* const part_a0 = sp.part;
  double* const part_col = sp.part + kServeMaxSlots * G;
  double* const part_row = sp.part + 2 * kServeMaxSlots * G;
  if (b == 0 && threadIdx.x < 32) serve_plan(sp, nullptr, &sp.st->plan[0], 0, sh);
  const bool started = grid_sync(base, target, sh);
  for (unsigned t = 0; started; ++t) {
    // this tick's plan, read past L1; the parameters of a slot change only
    // when a request is admitted, so they are copied in its first tick (and
    // for every slot at the start of a launch)
    {
      const int* src = reinterpret_cast<const int*>(&sp.st->plan[t & 1]);
      int* dst = reinterpret_cast<int*>(&plan);
      for (int e = threadIdx.x; e < static_cast<int>(sizeof(ServePlan) / 4); e += kThreads) dst[e] = __ldcg(src + e);
    }
    __syncthreads();
    {
      const int* ps = reinterpret_cast<const int*>(sp.st->p);
      int* pd = reinterpret_cast<int*>(prm);
      constexpr int kW = static_cast<int>(sizeof(Params) / 4);
      for (int s = 0; s < S; ++s)
        if (t == 0 || plan.col[s] == kColA0)
          for (int e = threadIdx.x; e < kW; e += kThreads) pd[s * kW + e] = __ldcg(ps + s * kW + e);
    }
    __syncthreads();
    // finish the previous tick: its row gaps, and the requests it completed
    if (t > 0 && b == 0 && threadIdx.x < 32) {
      const ServePlan& pp = sp.st->plan[(t - 1) & 1];
      for (int s = 0; s < S; ++s) {
        const int r = __ldcg(&pp.row[s]);
        if (r != kRowPass && r != kRowLast) continue;
        const double sum = serve_slot_sum(part_row + s * G, G);
        double* g_out = prm[s].g_out;  // unchanged until the slot is published
        if (threadIdx.x == 0 && g_out != nullptr) g_out[__ldcg(&pp.nu[s])] = sqrt(sum * prm[s].inv_n);
        if (threadIdx.x == 0 && r == kRowLast) serve_publish(sp.table, s, __ldcg(&sp.st->slot[s].seq), GS_OK);
      }
    }
    if (plan.stop) break;

    // column phase: A0 shares of admitted slots, column passes of running ones
    for (int s = 0; s < S; ++s)
      if (plan.col[s] == kColA0) serve_a0_partial(prm[s], part_a0 + s * G, sh);
    {
      int total = 0;  // column blocks of the running slots, one sequence split over the blocks
      for (int s = 0; s < S; ++s) total += (plan.col[s] == kColPass) ? (prm[s].nx >> 3) : 0;
      const int lo = G > 1 ? (b == 0 ? 0 : split(b - 1, G - 1, total)) : 0;
      const int hi = G > 1 ? (b == 0 ? 0 : split(b, G - 1, total)) : total;
      int k0 = 0;
      for (int s = 0; s < S; ++s) {
        if (plan.col[s] != kColPass) continue;
        const int units = prm[s].nx >> 3;
        const int slo = max(lo, k0) - k0, shi = min(hi, k0 + units) - k0;
        k0 += units;
        float a = 0.f;
        if (slo < shi) a = serve_run_pass(prm[s], kCol, false, slo, shi, smem, sh, mphase);
        const double tot = block_sum_f(a, sh);
        if (threadIdx.x == 0) part_col[s * G + b] = tot;
      }
    }
    if (!grid_sync(base, target, sh)) break;

    // scales of the admitted slots (every block, the same sums)
    for (int s = 0; s < S; ++s) {
      if (plan.col[s] != kColA0) continue;
      if (threadIdx.x < 32) {
        const double total = serve_slot_sum(part_a0 + s * G, G);
        if (threadIdx.x == 0) {
          const bool bad = !(total > 0.0) || !(total <= DBL_MAX);
          sh.bad[s] = bad ? 1 : 0;
          sh.scale[s] = bad ? 0.f : static_cast<float>(sqrt(static_cast<double>(prm[s].nx) * prm[s].ny / total));
          // the slot's amplitude is rebuilt: no column block of it stays resident
          sh.m_block = nullptr;
          sh.m_slot[0] = sh.m_slot[1] = nullptr;
        }
      }
      __syncthreads();
    }
    // r^nu of the running slots
    if (b == 0 && threadIdx.x < 32) {
      for (int s = 0; s < S; ++s) {
        if (plan.col[s] != kColPass) continue;
        const double sum = serve_slot_sum(part_col + s * G, G);
        if (threadIdx.x == 0 && prm[s].r_out != nullptr) prm[s].r_out[plan.nu[s]] = sqrt(sum * prm[s].inv_n);
      }
    }
    // row phase: m and the start of the admitted slots, row passes of the running ones
    for (int s = 0; s < S; ++s)
      if (plan.row[s] == kRowInit && !sh.bad[s]) build_amplitude(prm[s], 0, sh.scale[s], smem);
    {
      int total = 0;  // rows of the slots with row work, one sequence split over the blocks
      for (int s = 0; s < S; ++s)
        total += (plan.row[s] != kRowNone && !(plan.row[s] == kRowInit && sh.bad[s])) ? prm[s].ny : 0;
      const int lo = G > 1 ? (b == 0 ? 0 : split(b - 1, G - 1, total)) : 0;
      const int hi = G > 1 ? (b == 0 ? 0 : split(b, G - 1, total)) : total;
      int k0 = 0;
      for (int s = 0; s < S; ++s) {
        const int r = plan.row[s];
        if (r == kRowNone || (r == kRowInit && sh.bad[s])) continue;
        const int units = prm[s].ny;
        const int slo = max(lo, k0) - k0, shi = min(hi, k0 + units) - k0;
        k0 += units;
        const int kind = (r == kRowInit) ? kInit : kRow;
        float a = 0.f;
        if (slo < shi) {
          a = serve_run_pass(prm[s], kind, r == kRowLast, slo, shi, smem, sh, mphase);
          if (r == kRowLast) __threadfence_system();  // the phase in host memory before the publication
        }
        if (r != kRowInit) {
          const double tot = block_sum_f(a, sh);
          if (threadIdx.x == 0) part_row[s * G + b] = tot;
        }
      }
    }
    __syncthreads();
    if (b == 0 && threadIdx.x < 32) serve_plan(sp, &plan, &sp.st->plan[(t + 1) & 1], t + 1, sh);
    if (!grid_sync(base, target, sh)) break;
  }
  drain_copies(sh);
  if (b == 0 && threadIdx.x == 0) {
    st_volatile_i32(&sp.table->status, ld_volatile_i32(base.status));
    __threadfence_system();
    st_volatile_i32(&sp.table->running, 0);
    __threadfence_system();
  }
}

}  // namespace gsk
