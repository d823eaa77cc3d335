// gs_serve.cu -- the persistent server's C-ABI (include/gs.h): one cooperative
// launch of gs_serve (gs_serve.cuh) per serving period, a request table in
// pinned host memory, slot arrays in one device workspace.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "gs.h"
#include "gs_serve.cuh"

using gsk::kServeMaxSlots;
using gsk::ServeTable;

struct gs_server {
  int n = 0, L = 0, slots = 0, grid = 0;
  cudaStream_t stream = nullptr;
  unsigned char* ws = nullptr;  // device workspace
  ServeTable* table = nullptr;  // pinned, mapped host memory
  gsk::ServeParams sp{};
  cudaEvent_t ev = nullptr;     // recorded after each launch
  bool launched = false;
  unsigned next_seq = 0;
  unsigned posted[kServeMaxSlots] = {};
  size_t smem = 0;
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

const void* serve_kernel() { return reinterpret_cast<const void*>(gsk::gs_serve); }

unsigned load_u32(const unsigned* a) { return __atomic_load_n(a, __ATOMIC_ACQUIRE); }
int load_i32(const int* a) { return __atomic_load_n(a, __ATOMIC_ACQUIRE); }

bool outstanding(const gs_server* s) {
  for (int k = 0; k < s->slots; ++k)
    if (load_u32(&s->table->done_seq[k]) != s->posted[k]) return true;
  return false;
}

// A launch serves while `running` is set; a launch that left (idle, tick
// limit, stop) has cleared it. Relaunch when requests are outstanding and no
// launch is running or queued.
int ensure_running(gs_server* s) {
  if (load_i32(&s->table->status) != GS_OK) return load_i32(&s->table->status);
  if (load_i32(&s->table->running) != 0) return GS_OK;
  if (s->launched && cudaEventQuery(s->ev) == cudaErrorNotReady) return GS_OK;  // still leaving, or queued
  cudaGetLastError();
  __atomic_store_n(&s->table->running, 1, __ATOMIC_SEQ_CST);
  void* args[] = {&s->sp};
  if (cudaMemsetAsync(s->sp.base.bar, 0, sizeof(unsigned), s->stream) != cudaSuccess ||
      cudaLaunchCooperativeKernel(serve_kernel(), dim3(s->grid), dim3(gsk::kThreads), args, s->smem, s->stream) !=
          cudaSuccess ||
      cudaEventRecord(s->ev, s->stream) != cudaSuccess) {
    cudaGetLastError();
    __atomic_store_n(&s->table->running, 0, __ATOMIC_SEQ_CST);
    return GS_ECUDA;
  }
  s->launched = true;
  return GS_OK;
}

}  // namespace

extern "C" {

int gs_serve_create(gs_server** out, int max_n, int slots, int grid, void* stream) {
  if (out == nullptr) return GS_EINVAL;
  *out = nullptr;
  const int n = max_n;
  int L = 0;
  while ((1 << L) < n) ++L;
  if ((1 << L) != n || L < 8 || L > 10 || slots < 1 || slots > kServeMaxSlots || grid < 0) return GS_EINVAL;
  gs_server* s = new (std::nothrow) gs_server;
  if (s == nullptr) return GS_ENOMEM;
  s->n = n;
  s->L = L;
  s->slots = slots;
  s->stream = static_cast<cudaStream_t>(stream);
  s->smem = static_cast<size_t>(gsk::kGroupSmemBytes) + 8192 * 4 + 8192 * 8;
  int dev = 0, sms = 0, per_sm = 0;
  const void* k = serve_kernel();
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(s->smem)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, gsk::kThreads, s->smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    delete s;
    return GS_ECUDA;
  }
  const int cap = sms * per_sm < gsk::kMaxGrid ? sms * per_sm : gsk::kMaxGrid;
  s->grid = grid > 0 ? grid : cap;
  if (s->grid > cap) s->grid = cap;

  const size_t npix = static_cast<size_t>(n) * n;
  size_t o = 0;
  const size_t oB = o;    o = align_up(o + slots * npix * sizeof(float2));
  const size_t omT = o;   o = align_up(o + slots * npix * sizeof(float));
  const size_t opart = o; o = align_up(o + 3 * static_cast<size_t>(kServeMaxSlots) * s->grid * sizeof(double));
  const size_t otw = o;   o = align_up(o + 3 * static_cast<size_t>(gsk::kStageTwiddleEntries) * sizeof(float2));
  const size_t oones = o; o = align_up(o + 4096 * sizeof(float));
  const size_t obar = o;  o = align_up(o + sizeof(unsigned));
  const size_t ostat = o; o = align_up(o + sizeof(int));
  const size_t oabort = o; o = align_up(o + sizeof(int));
  const size_t oflags = o; o = align_up(o + kServeMaxSlots * sizeof(int));
  const size_t ost = o;   o = align_up(o + sizeof(gsk::ServeState));
  std::vector<float2> tw(3 * static_cast<size_t>(gsk::kStageTwiddleEntries));
  for (int k = 0; 8 + k <= L; ++k) gsk::stage_twiddles_host(256 << k, tw.data() + k * gsk::kStageTwiddleEntries);
  const std::vector<float> ones(4096, 1.0f);
  if (cudaMalloc(&s->ws, o) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return GS_ENOMEM;
  }
  if (cudaHostAlloc(&s->table, sizeof(ServeTable), cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->ws);
    delete s;
    return GS_ENOMEM;
  }
  std::memset(s->table, 0, sizeof(ServeTable));
  ServeTable* dtab = nullptr;
  bool ok = cudaHostGetDevicePointer(reinterpret_cast<void**>(&dtab), s->table, 0) == cudaSuccess &&
            cudaMemset(s->ws, 0, o) == cudaSuccess &&
            cudaMemcpy(s->ws + otw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(s->ws + oones, ones.data(), ones.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaFreeHost(s->table);
    cudaFree(s->ws);
    delete s;
    return GS_ECUDA;
  }
  gsk::Params& p = s->sp.base;
  std::memset(&p, 0, sizeof(p));
  p.nx = p.ny = n;
  p.lognx = p.logny = L;
  p.B = reinterpret_cast<float2*>(s->ws + oB);
  p.mT = reinterpret_cast<float*>(s->ws + omT);
  p.partials = reinterpret_cast<double*>(s->ws + opart);
  for (int k = 0; k < 3; ++k)
    s->sp.tw[k] = 8 + k <= L ? reinterpret_cast<const float2*>(s->ws + otw) + k * gsk::kStageTwiddleEntries : nullptr;
  s->sp.max_log = L;
  s->sp.max_ticks = gsk::kServeMaxTicks;
  p.ones = reinterpret_cast<const float*>(s->ws + oones);
  p.bar = reinterpret_cast<unsigned*>(s->ws + obar);
  p.status = reinterpret_cast<int*>(s->ws + ostat);
  p.abort_flag = reinterpret_cast<int*>(s->ws + oabort);
  p.mask_flags = reinterpret_cast<int*>(s->ws + oflags);
  p.batch = 1;
  p.mstride = static_cast<long long>(npix);
  p.rstride = p.gstride = 0;
  p.group = 1;
  const double nn = static_cast<double>(npix);
  p.inv_sqrt_n = static_cast<float>(1.0 / std::sqrt(nn));
  p.inv_n = 1.0 / nn;
  s->sp.table = dtab;
  s->sp.st = reinterpret_cast<gsk::ServeState*>(s->ws + ost);
  s->sp.part = reinterpret_cast<double*>(s->ws + opart);
  s->sp.slots = slots;
  *out = s;
  return GS_OK;
}

int gs_serve_submit(gs_server* s, int slot, int n, const float* target_intensity, const float* phase_in,
                    int iters, float* phase_out, double* residual_out, double* object_gap_out, unsigned* seq_out) {
  if (s == nullptr || slot < 0 || slot >= s->slots || iters < 1 || target_intensity == nullptr ||
      phase_in == nullptr || phase_out == nullptr || !(n == 256 || n == 512 || n == 1024) || n > s->n)
    return GS_EINVAL;
  if (load_u32(&s->table->done_seq[slot]) != s->posted[slot]) return GS_EINVAL;  // the slot is busy
  // every buffer must be pinned host memory the device can address
  const void* bufs[5] = {target_intensity, phase_in, phase_out, residual_out, object_gap_out};
  void* dp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int k = 0; k < 5; ++k) {
    if (bufs[k] == nullptr) continue;
    if (cudaHostGetDevicePointer(&dp[k], const_cast<void*>(bufs[k]), 0) != cudaSuccess) {
      cudaGetLastError();
      return GS_EINVAL;
    }
  }
  gsk::ServeRequest& q = s->table->req[slot];
  q.I = static_cast<const float*>(dp[0]);
  q.phi_in = static_cast<const float*>(dp[1]);
  q.phi_out = static_cast<float*>(dp[2]);
  q.r_out = static_cast<double*>(dp[3]);
  q.g_out = static_cast<double*>(dp[4]);
  q.K = iters;
  q.n = n;
  unsigned seq = ++s->next_seq;
  if (seq == 0) seq = ++s->next_seq;  // 0 is the initial value of every slot
  s->posted[slot] = seq;
  __atomic_store_n(&s->table->req_seq[slot], seq, __ATOMIC_RELEASE);
  std::atomic_thread_fence(std::memory_order_seq_cst);
  if (seq_out) *seq_out = seq;
  return ensure_running(s);
}

int gs_serve_poll(gs_server* s, int slot, unsigned* done_seq, int* request_status) {
  if (s == nullptr || slot < 0 || slot >= s->slots) return GS_EINVAL;
  const unsigned d = load_u32(&s->table->done_seq[slot]);
  if (done_seq) *done_seq = d;
  if (request_status) *request_status = load_i32(&s->table->done_status[slot]);
  if (d != s->posted[slot] || outstanding(s)) return ensure_running(s);
  return load_i32(&s->table->status);
}

int gs_serve_stop(gs_server* s) {
  if (s == nullptr) return GS_EINVAL;
  // let the running launch finish its requests and leave; relaunch while
  // requests are outstanding and the server has not failed
  __atomic_store_n(&s->table->stop, 1, __ATOMIC_SEQ_CST);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60)) {  // requests that never finish
      __atomic_store_n(&s->table->stop, 0, __ATOMIC_SEQ_CST);
      return GS_ETIMEOUT;
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
      cudaGetLastError();
      return GS_ECUDA;
    }
    const int st = load_i32(&s->table->status);
    if (st != GS_OK || !outstanding(s)) break;
    __atomic_store_n(&s->table->stop, 0, __ATOMIC_SEQ_CST);
    const int rc = ensure_running(s);
    __atomic_store_n(&s->table->stop, 1, __ATOMIC_SEQ_CST);
    if (rc != GS_OK) return rc;
  }
  __atomic_store_n(&s->table->stop, 0, __ATOMIC_SEQ_CST);
  return load_i32(&s->table->status);
}

int gs_serve_grid(const gs_server* s) { return s ? s->grid : 0; }

int gs_serve_test_tick_limit(gs_server* s, int ticks) {
  if (s == nullptr || ticks < 1 || static_cast<unsigned>(ticks) > gsk::kServeMaxTicks) return GS_EINVAL;
  if (load_i32(&s->table->running) != 0 || (s->launched && cudaEventQuery(s->ev) == cudaErrorNotReady)) {
    cudaGetLastError();
    return GS_EINVAL;  // only between launches
  }
  s->sp.max_ticks = static_cast<unsigned>(ticks);
  return GS_OK;
}

void gs_serve_destroy(gs_server* s) {
  if (s == nullptr) return;
  gs_serve_stop(s);
  cudaStreamSynchronize(s->stream);
  if (s->ev) cudaEventDestroy(s->ev);
  cudaFreeHost(s->table);
  cudaFree(s->ws);
  cudaGetLastError();
  delete s;
}

}  // extern "C"
