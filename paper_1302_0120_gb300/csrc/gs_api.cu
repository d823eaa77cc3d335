// gs_api.cu -- the C ABI: context, workspace, validation and launches.
//
// Host code only. Every entry point validates its arguments before touching
// CUDA, returns a GS_* status and lets no exception escape.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "gs.h"
#include "gs_internal.h"

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// 2^a 3^b 5^c
bool smooth5(int n) {
  if (n < 1) return false;
  for (int f : {2, 3, 5})
    while (n % f == 0) n /= f;
  return n == 1;
}

// A grid side: a power of two in [8, 4096], or a 5-smooth number in
// [8, kMaxGeneralSide] (sides that are not powers of two, or below 32, run on
// the general kernel).
bool valid_dim(int n) {
  if (n < 8) return false;
  if (is_pow2(n)) return n <= 4096;
  return n <= gsk::kMaxGeneralSide && smooth5(n);
}

// Radix plan of a 5-smooth length for the general kernel: radices 3 and 5
// first (their unit-stride reads and odd-stride writes stay free of bank
// conflicts while the sub-transforms are short), then 8s, then a 4 or 2.
// Code c of stage s sits in bits 3s..3s+2 (2 -> 0, 3 -> 1, 4 -> 2, 5 -> 3, 8 -> 4).
void radix_plan(int n, unsigned* plan, int* nst) {
  std::vector<int> r;
  while (n % 3 == 0) { r.push_back(3); n /= 3; }
  while (n % 5 == 0) { r.push_back(5); n /= 5; }
  while (n % 8 == 0) { r.push_back(8); n /= 8; }
  if (n == 4) r.push_back(4);
  if (n == 2) r.push_back(2);
  unsigned code = 0;  // 3 bits per stage; 5-smooth sides up to kMaxGeneralSide need at most 7 stages
  static_assert(3 * gsk::kMaxGeneralStages <= 32, "stage codes fit the plan word");
  if (r.size() > static_cast<size_t>(gsk::kMaxGeneralStages)) r.resize(0);  // unreachable for valid sides
  for (size_t s = 0; s < r.size(); ++s) {
    const unsigned c = r[s] == 2 ? 0u : r[s] == 3 ? 1u : r[s] == 4 ? 2u : r[s] == 5 ? 3u : 4u;
    code |= c << (3 * s);
  }
  *plan = code;
  *nst = static_cast<int>(r.size());
}

int ilog2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Entries of one stage-twiddle table (stages after 32 and after 1024 points).
constexpr int kTwiddleEntries = gsk::kStageTwiddleEntries;

// Offsets of the sub-buffers of one workspace allocation.
struct Layout {
  size_t B, mT, partials, twx, twy, ones, bar, status, abort_flag, mask_flags, energy, lossbuf, dI, dphi, trace, total;
  size_t guard[16];  // canary words after each buffer (gs_check_workspace)
  int nguard;
};

constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;

Layout make_layout(int nx, int ny, int max_batch) {
  const size_t n = static_cast<size_t>(nx) * ny;
  const size_t nb = n * static_cast<size_t>(max_batch);
  Layout L{};
  size_t o = 0;
  L.B = o;          o = align_up(o + nb * sizeof(float2));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.mT = o;         o = align_up(o + nb * sizeof(float));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.partials = o;
  o = align_up(o + static_cast<size_t>(gsk::kSlots) * max_batch * gsk::kMaxGrid * sizeof(double));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.twx = o;        o = align_up(o + static_cast<size_t>(kTwiddleEntries) * sizeof(float2));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.twy = o;        o = align_up(o + static_cast<size_t>(kTwiddleEntries) * sizeof(float2));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.ones = o;       o = align_up(o + 4096 * sizeof(float));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  // the barrier counter and the abort word side by side: one memset clears
  // both before the first launch of a run
  L.bar = o;
  L.abort_flag = o + sizeof(unsigned);
  o = align_up(o + 2 * sizeof(unsigned));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.status = o;     o = align_up(o + sizeof(int));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.mask_flags = o; o = align_up(o + gsk::kMaxBatch * sizeof(int));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.energy = o;     o = align_up(o + sizeof(double));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.lossbuf = o;    o = align_up(o + sizeof(double));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.dI = o;         o = align_up(o + n * sizeof(float));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.dphi = o;       o = align_up(o + n * sizeof(float));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.trace = o;      o = align_up(o + static_cast<size_t>(gsk::kTraceRows) * gsk::kMaxGrid * 2 * sizeof(unsigned long long));
  L.guard[L.nguard++] = o; o += kGuardBytes;
  L.total = o;
  return L;
}

// exp(-2 pi i k / M) computed in double and rounded once; points on the eight
// octant directions are exact.
float2 unit_root(long long k, long long M) {
  k %= M;
  if ((8 * k) % M == 0) {
    const double h = std::sqrt(0.5);
    const double oc[8] = {1.0, h, 0.0, -h, -1.0, -h, 0.0, h};
    const double os[8] = {0.0, h, 1.0, h, 0.0, -h, -1.0, -h};
    const int o = static_cast<int>((8 * k) / M);
    return make_float2(static_cast<float>(oc[o]), static_cast<float>(-os[o]));
  }
  const double a = 2.0 * M_PI * static_cast<double>(k) / static_cast<double>(M);
  return make_float2(static_cast<float>(std::cos(a)), static_cast<float>(-std::sin(a)));
}

// Stage twiddle tables of a length-n transform, in the layout stage_c reads:
// for the stage after Ns = 2^nsl points (nsl = 5, 10) with radix R, entry
// offset(nsl) + (m - 1) Ns + r holds W_{Ns R}^{r m}.
// The general kernel (a side that is not a power of two) reads instead, for
// both sides, the stage tables of its radix plan: the stage with
// sub-transform length ns and radix R holds W_{ns R}^{r m} at entry
// ns - 1 + (m - 1) ns + r (1 <= m < R, r < ns); n - 1 entries in all.
// Tables of the register-resident kernel (gs_rg.cuh) for a side n = T V:
// W_n^{t q} at [q T + t] (q < V, t < T), then W_n^{q j} at n + [j V + q].
std::vector<float2> rg_twiddles(int n) {
  std::vector<float2> w(kTwiddleEntries, make_float2(0.f, 0.f));
  const int T = gsk::rg_threads(n), V = n / T;
  for (int q = 0; q < V; ++q)
    for (int t = 0; t < T; ++t) w[q * T + t] = unit_root(static_cast<long long>(t) * q, n);
  for (int j = 0; j < T; ++j)
    for (int q = 0; q < V; ++q) w[n + j * V + q] = unit_root(static_cast<long long>(q) * j, n);
  return w;
}

std::vector<float2> twiddles(int n, bool general) {
  std::vector<float2> w(kTwiddleEntries, make_float2(0.f, 0.f));
  if (general) {
    unsigned plan = 0;
    int nst = 0;
    radix_plan(n, &plan, &nst);
    int ns = 1;
    for (int s = 0; s < nst; ++s) {
      const unsigned c = (plan >> (3 * s)) & 7u;
      const int R = c == 0 ? 2 : c == 1 ? 3 : c == 2 ? 4 : c == 3 ? 5 : 8;
      for (int m = 1; m < R; ++m)
        for (int r = 0; r < ns; ++r)
          w[ns - 1 + (m - 1) * ns + r] = unit_root(static_cast<long long>(r) * m, static_cast<long long>(ns) * R);
      ns *= R;
    }
    return w;
  }
  for (int nsl = 5; nsl < 12; nsl += 5) {
    const int ns = 1 << nsl;
    if (n <= ns) break;
    int R = n / ns;
    if (R > 32) R = 32;
    const int off = nsl == 5 ? 0 : 31 * 32;
    for (int m = 1; m < R; ++m)
      for (int r = 0; r < ns; ++r) w[off + (m - 1) * ns + r] = unit_root(static_cast<long long>(r) * m, static_cast<long long>(ns) * R);
  }
  return w;
}

}  // namespace

struct gs_ctx {
  int nx = 0, ny = 0;
  int max_batch = 1;
  unsigned flags = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  int blocks_per_sm = 0;
  int grid_override = 0;
  int tc_mode = 0;               // gsk::TcMode of the iteration kernel
  bool loss_prepared = false;    // the workspace holds a target staged by gs_loss_prepare
  const float* p_slm = nullptr;  // caller-owned SLM amplitude, or null (p = 1)
  unsigned extra_arrivals = 0;
  int group_override = 0;  // masks per group of a batched run (0: the whole batch)
  bool trace = false;      // record pass timestamps (gs_set_trace)
  int trace_grid = 0, trace_passes = 0;  // shape of the last traced launch
  Layout L{};
  unsigned char* ws = nullptr;
  double* dres = nullptr;  // device residual staging for gs_run_host
  double* hres = nullptr;  // pinned host copy of it, plus a word for the status
  size_t dres_cap = 0;     // doubles
  // gs_create_mixed: one workspace per size class n = 256 << k (max_batch > 0),
  // at byte offset mbase[k]; L above is the first such class, at offset 0.
  bool mixed = false;
  int mixed_max[3] = {0, 0, 0};
  Layout Lm[3]{};
  size_t mbase[3] = {0, 0, 0};
};

namespace {

template <typename T>
T* at(gs_ctx* c, size_t off) {
  return reinterpret_cast<T*>(c->ws + off);
}

int max_grid(const gs_ctx* c) {
  int m = c->num_sms * c->blocks_per_sm;
  if (m > gsk::kMaxGrid) m = gsk::kMaxGrid;
  return m < 1 ? 1 : m;
}

int choose_grid_for(const gs_ctx* c, long long pixels) {
  const int cap = max_grid(c);
  int g;
  if (c->grid_override > 0) {
    g = c->grid_override;
  } else {
    // one block per 4096 pixels; small grids get up to 32 blocks (one per
    // 2048 pixels): there the passes are latency-bound and more blocks
    // shorten each block's share (measured on 256 x 256: 1.61 -> 1.34 ms per
    // 100 iterations)
    const long long n = pixels;
    g = static_cast<int>(n / 4096);
    const int small = static_cast<int>(n / 2048 < 32 ? n / 2048 : 32);
    if (g < small) g = small;
  }
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return g;
}

// Masks iterated together: by default as many as keep their fields (B, 8
// bytes per pixel, and m, 4) within kGroupBytes, so that a group stays in L2
// while it runs the schedule; the caller can fix the size instead. Measured
// on one GB300 (50 iterations): 8 x 1024^2 (96 MiB) is fastest in one group
// (0.58 ms per mask, 0.65 in groups of 5), 16 x 1024^2 in groups of 8 (0.58 vs
// 0.62 in one group), 32 x 512^2 in groups of 16 or 32 (0.31-0.33).
constexpr long long kGroupBytes = 100ll << 20;

int group_size(const gs_ctx* c, long long pixels, int batch) {
  long long g = c->group_override > 0 ? c->group_override : kGroupBytes / (12 * pixels);
  if (g < 1) g = 1;
  return static_cast<int>(g < batch ? g : batch);
}

// Fill (or check) the canary words of one workspace layout at ws.
bool fill_guards(unsigned char* ws, const Layout& L) {
  for (int g = 0; g < L.nguard; ++g)
    if (cudaMemset(ws + L.guard[g], kGuardByte, kGuardBytes) != cudaSuccess) return false;
  return true;
}

int check_guards(const unsigned char* ws, const Layout& L) {
  unsigned char h[kGuardBytes];
  for (int g = 0; g < L.nguard; ++g) {
    if (cudaMemcpy(h, ws + L.guard[g], kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return GS_ECUDA;
    }
    for (size_t k = 0; k < kGuardBytes; ++k)
      if (h[k] != kGuardByte) return GS_ECORRUPT;
  }
  return GS_OK;
}

int choose_grid(const gs_ctx* c) {
  if (!c->mixed && gsk::uses_general(c->nx, c->ny) && !gsk::uses_rg(c->nx, c->ny) && c->grid_override <= 0) {
    // general sides: one row per team (four per block) and one 4-column
    // group per block, so that each pass is one round
    const int t = gsk::kGenTeams;
    int g = (c->ny + t - 1) / t;
    const int gc = (c->nx + t - 1) / t;
    if (gc > g) g = gc;
    const int cap = max_grid(c);
    return g > cap ? cap : g;
  }
  return choose_grid_for(c, static_cast<long long>(c->nx) * c->ny);
}

}  // namespace

namespace gsk {
void stage_twiddles_host(int n, float2* out) {
  const std::vector<float2> w = twiddles(n, false);
  std::copy(w.begin(), w.end(), out);
}
}  // namespace gsk

extern "C" {

const char* gs_strerror(int code) {
  switch (code) {
    case GS_OK: return "success";
    case GS_EINVAL: return "invalid argument";
    case GS_ENOMEM: return "out of memory";
    case GS_ECUDA: return "CUDA runtime error";
    case GS_ETIMEOUT: return "device-side wait timed out";
    case GS_ENUMERIC: return "target intensity is non-finite, negative or zero";
    case GS_ECORRUPT: return "a canary word of the workspace was overwritten";
    default: return "unknown status";
  }
}

size_t gs_workspace_bytes_batched(int nx, int ny, int max_batch, unsigned flags) {
  (void)flags;
  if (!valid_dim(nx) || !valid_dim(ny) || max_batch < 1 || max_batch > gsk::kMaxBatch) return 0;
  return make_layout(nx, ny, max_batch).total;
}

size_t gs_workspace_bytes(int nx, int ny, unsigned flags) { return gs_workspace_bytes_batched(nx, ny, 1, flags); }

int gs_create(gs_ctx** out, int nx, int ny, unsigned flags, void* stream) {
  return gs_create_batched(out, nx, ny, 1, flags, stream);
}

int gs_create_batched(gs_ctx** out, int nx, int ny, int max_batch, unsigned flags, void* stream) {
  if (out == nullptr) return GS_EINVAL;
  *out = nullptr;
  if (!valid_dim(nx) || !valid_dim(ny) || max_batch < 1 || max_batch > gsk::kMaxBatch) return GS_EINVAL;
  if ((flags & ~static_cast<unsigned>(GS_FINAL_RESIDUAL | GS_INIT_FROM_TARGET | GS_TENSOR_CORE | GS_BF16 |
                                      GS_TC_MMA_SYNC)) != 0)
    return GS_EINVAL;
  const bool tc = (flags & GS_TENSOR_CORE) != 0;
  if (tc && !(nx == ny && is_pow2(nx) && nx >= 256 && nx <= 1024)) return GS_EINVAL;
  if ((flags & (GS_BF16 | GS_TC_MMA_SYNC)) != 0 && !tc) return GS_EINVAL;
  // the transforms run through tcgen05 unless mma.sync is asked for (FP16
  // operands only)
  const bool tc5 = tc && !(flags & GS_TC_MMA_SYNC);
  if ((flags & GS_BF16) != 0 && !tc5) return GS_EINVAL;
  const int tc_mode = !tc ? gsk::kTcNone : !tc5 ? gsk::kTcMmaSync : (flags & GS_BF16) ? gsk::kTcGen05Bf16 : gsk::kTcGen05F16;
  gs_ctx* c = new (std::nothrow) gs_ctx();
  if (c == nullptr) return GS_ENOMEM;
  c->tc_mode = tc_mode;
  c->nx = nx;
  c->ny = ny;
  c->max_batch = max_batch;
  c->flags = flags;
  c->stream = static_cast<cudaStream_t>(stream);
  c->L = make_layout(nx, ny, max_batch);
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
      gsk::iteration_occupancy(nx, ny, &c->blocks_per_sm, tc_mode) != cudaSuccess || c->blocks_per_sm < 1 ||
      (gsk::small_grid(nx, ny) && gsk::small_prepare(nx, ny) != cudaSuccess)) {
    cudaGetLastError();
    delete c;
    return GS_ECUDA;
  }
  if (cudaMalloc(&c->ws, c->L.total) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return GS_ENOMEM;
  }
  const bool general = gsk::uses_general(nx, ny);
  const bool rg = gsk::uses_rg(nx, ny);
  const std::vector<float2> wx = rg ? rg_twiddles(nx) : twiddles(nx, general);
  const std::vector<float2> wy = rg ? rg_twiddles(ny) : twiddles(ny, general);
  const std::vector<float> ones(4096, 1.0f);
  bool ok = cudaMemcpy(c->ws + c->L.twx, wx.data(), wx.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->ws + c->L.ones, ones.data(), ones.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->ws + c->L.twy, wy.data(), wy.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(c->ws + c->L.bar, 0, c->L.dI - c->L.bar) == cudaSuccess && fill_guards(c->ws, c->L);
  if (!ok) {
    cudaGetLastError();
    cudaFree(c->ws);
    delete c;
    return GS_ECUDA;
  }
  *out = c;
  return GS_OK;
}

int gs_run(gs_ctx* c, const float* target_intensity, const float* phase_in, int iters, float* phase_out,
           double* residual_out, double* object_gap_out) {
  return gs_run_batched(c, 1, target_intensity, phase_in, iters, phase_out, residual_out, object_gap_out);
}

int gs_run_batched(gs_ctx* c, int batch, const float* target_intensity, const float* phase_in, int iters,
                   float* phase_out, double* residual_out, double* object_gap_out) {
  const bool from_target = (c != nullptr) && (c->flags & GS_INIT_FROM_TARGET);
  if (c == nullptr || c->mixed || target_intensity == nullptr || (phase_in == nullptr && !from_target) ||
      phase_out == nullptr || iters < 0 || batch < 1 || batch > c->max_batch)
    return GS_EINVAL;
  // Small grids run one block per mask with the field in shared memory,
  // unless a fixed grid, a variant the small kernel does not implement (the
  // target start, a laser amplitude, tensor cores) or a diagnostic (pass
  // timestamps, the barrier test hook) asks for the persistent kernel.
  const bool small = gsk::small_grid(c->nx, c->ny) && c->grid_override == 0 && !from_target &&
                     c->p_slm == nullptr && !(c->flags & GS_TENSOR_CORE) && !c->trace && c->extra_arrivals == 0;
  const int grid = choose_grid(c);
  c->loss_prepared = false;  // the run's amplitude overwrites a staged loss target
  gsk::Params p{};
  p.batch = batch;
  p.mstride = static_cast<long long>(c->nx) * c->ny;
  p.rstride = iters + ((c->flags & GS_FINAL_RESIDUAL) ? 1 : 0);
  p.gstride = iters;
  p.nx = c->nx;
  p.ny = c->ny;
  p.lognx = ilog2i(c->nx);
  p.logny = ilog2i(c->ny);
  radix_plan(c->nx, &p.planx, &p.nstx);
  radix_plan(c->ny, &p.plany, &p.nsty);
  p.B = at<float2>(c, c->L.B);
  p.mT = at<float>(c, c->L.mT);
  p.I = target_intensity;
  p.phi_in = phase_in;
  p.phi_out = phase_out;
  p.partials = at<double>(c, c->L.partials);
  p.r_out = residual_out;
  p.g_out = object_gap_out;
  p.twx = at<float2>(c, c->L.twx);
  p.twy = at<float2>(c, c->L.twy);
  p.bar = at<unsigned>(c, c->L.bar);
  p.status = at<int>(c, c->L.status);
  p.abort_flag = at<int>(c, c->L.abort_flag);
  p.mask_flags = at<int>(c, c->L.mask_flags);
  p.p_slm = c->p_slm;
  p.energy = at<double>(c, c->L.energy);
  p.ones = at<float>(c, c->L.ones);
  p.init_target = from_target ? 1 : 0;
  p.iters = iters;
  p.final_resid = (c->flags & GS_FINAL_RESIDUAL) ? 1 : 0;
  p.extra_arrivals = c->extra_arrivals;
  p.tensor_core = c->tc_mode;
  p.group = group_size(c, static_cast<long long>(c->nx) * c->ny, batch);
  p.trace = c->trace ? at<unsigned long long>(c, c->L.trace) : nullptr;
  const double n = static_cast<double>(c->nx) * c->ny;
  p.inv_sqrt_n = static_cast<float>(1.0 / std::sqrt(n));
  p.inv_n = 1.0 / n;
  if (small) {  // one launch for the whole run, whatever K
    p.it0 = 0;
    p.it1 = iters;
    p.do_init = p.do_final = 1;
    if (gsk::launch_small(p, c->stream) != cudaSuccess) {
      cudaGetLastError();
      return GS_ECUDA;
    }
    return GS_OK;
  }
  int it0 = 0;
  do {
    int it1 = it0 + gsk::kMaxIterPerLaunch;
    if (it1 > iters) it1 = iters;
    p.it0 = it0;
    p.it1 = it1;
    p.do_init = (it0 == 0) ? 1 : 0;
    p.do_final = (it1 == iters) ? 1 : 0;
    // the barrier counter before every launch; the abort word (next to it)
    // before the first one only, so that a failed launch stops the later ones
    if (cudaMemsetAsync(p.bar, 0, (it0 == 0 ? 2 : 1) * sizeof(unsigned), c->stream) != cudaSuccess ||
        gsk::launch_iterations(p, grid, c->stream) != cudaSuccess) {
      cudaGetLastError();
      return GS_ECUDA;
    }
    it0 = it1;
  } while (it0 < iters);
  if (c->trace) {  // the shape of the last launch's record
    c->trace_grid = grid;
    c->trace_passes = (p.do_init ? (p.init_target ? 2 : 1) : 0) + 2 * (p.it1 - p.it0) +
                      ((p.do_final && p.final_resid) ? 1 : 0);
  }
  return GS_OK;
}

int gs_create_mixed(gs_ctx** out, const int* max_batch, unsigned flags, void* stream) {
  if (out == nullptr) return GS_EINVAL;
  *out = nullptr;
  if (max_batch == nullptr) return GS_EINVAL;
  int total = 0;
  for (int k = 0; k < 3; ++k) {
    if (max_batch[k] < 0 || max_batch[k] > gsk::kMaxBatch) return GS_EINVAL;
    total += max_batch[k];
  }
  if (total < 1 || total > gsk::kMaxBatch) return GS_EINVAL;
  if ((flags & ~static_cast<unsigned>(GS_FINAL_RESIDUAL | GS_INIT_FROM_TARGET | GS_TENSOR_CORE | GS_BF16 |
                                      GS_TC_MMA_SYNC)) != 0)
    return GS_EINVAL;
  const bool tc = (flags & GS_TENSOR_CORE) != 0;
  if ((flags & (GS_BF16 | GS_TC_MMA_SYNC)) != 0 && !tc) return GS_EINVAL;
  if ((flags & GS_BF16) != 0 && (flags & GS_TC_MMA_SYNC) != 0) return GS_EINVAL;
  const int tc_mode = !tc ? gsk::kTcNone
                      : (flags & GS_TC_MMA_SYNC) ? gsk::kTcMmaSync
                      : (flags & GS_BF16) ? gsk::kTcGen05Bf16
                                          : gsk::kTcGen05F16;
  gs_ctx* c = new (std::nothrow) gs_ctx();
  if (c == nullptr) return GS_ENOMEM;
  c->tc_mode = tc_mode;
  c->mixed = true;
  c->flags = flags;
  c->stream = static_cast<cudaStream_t>(stream);
  size_t off = 0;
  int primary = -1;
  for (int k = 0; k < 3; ++k) {
    c->mixed_max[k] = max_batch[k];
    if (max_batch[k] == 0) continue;
    const int n = 256 << k;
    if (primary < 0) primary = k;
    c->Lm[k] = make_layout(n, n, max_batch[k]);
    c->mbase[k] = off;
    off += c->Lm[k].total;
  }
  c->L = c->Lm[primary];
  c->nx = c->ny = 256 << primary;
  c->max_batch = total;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
      gsk::mixed_occupancy(tc_mode, &c->blocks_per_sm) != cudaSuccess || c->blocks_per_sm < 1) {
    cudaGetLastError();
    delete c;
    return GS_ECUDA;
  }
  if (cudaMalloc(&c->ws, off) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return GS_ENOMEM;
  }
  bool ok = true;
  for (int k = 0; k < 3 && ok; ++k) {
    if (max_batch[k] == 0) continue;
    const Layout& L = c->Lm[k];
    unsigned char* w = c->ws + c->mbase[k];
    const std::vector<float2> tw = twiddles(256 << k, false);
    ok = cudaMemcpy(w + L.twx, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(w + L.twy, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(w + L.bar, 0, L.dI - L.bar) == cudaSuccess && fill_guards(w, L);
  }
  if (!ok) {
    cudaGetLastError();
    cudaFree(c->ws);
    delete c;
    return GS_ECUDA;
  }
  *out = c;
  return GS_OK;
}

int gs_run_mixed(gs_ctx* c, const int* batch, const float* const* target_intensity, const float* const* phase_in,
                 int iters, float* const* phase_out, double* const* residual_out, double* const* object_gap_out) {
  if (c == nullptr || !c->mixed || batch == nullptr || target_intensity == nullptr || phase_out == nullptr ||
      iters < 0)
    return GS_EINVAL;
  const bool from_target = (c->flags & GS_INIT_FROM_TARGET) != 0;
  if (phase_in == nullptr && !from_target) return GS_EINVAL;
  int total = 0;
  for (int k = 0; k < 3; ++k) {
    if (batch[k] < 0 || batch[k] > c->mixed_max[k]) return GS_EINVAL;
    if (batch[k] > 0 && (target_intensity[k] == nullptr || phase_out[k] == nullptr ||
                         (!from_target && phase_in[k] == nullptr)))
      return GS_EINVAL;
    total += batch[k];
  }
  if (total < 1) return GS_EINVAL;
  int largest = 0;
  for (int k = 0; k < 3; ++k)
    if (batch[k] > 0) largest = k;
  const long long px = static_cast<long long>(256 << largest) * (256 << largest);
  const int grid = choose_grid_for(c, px);  // the single-size rule for the largest class present
  const Layout& P = c->L;  // the primary class holds the barrier, status and abort words
  unsigned char* const pw = c->ws;
  gsk::MixedParams mp{};
  for (int k = 0; k < 3; ++k) {
    gsk::Params& p = mp.cls[k];
    const int n = 256 << k;
    p.nx = p.ny = n;
    p.lognx = p.logny = 8 + k;
    p.batch = batch[k];
    p.mstride = static_cast<long long>(n) * n;
    p.rstride = iters + ((c->flags & GS_FINAL_RESIDUAL) ? 1 : 0);
    p.gstride = iters;
    p.iters = iters;
    p.final_resid = (c->flags & GS_FINAL_RESIDUAL) ? 1 : 0;
    p.init_target = from_target ? 1 : 0;
    p.extra_arrivals = c->extra_arrivals;
    p.tensor_core = c->tc_mode;
    p.group = group_size(c, static_cast<long long>(n) * n, batch[k] > 0 ? batch[k] : 1);
    p.inv_sqrt_n = static_cast<float>(1.0 / n);
    p.inv_n = 1.0 / (static_cast<double>(n) * n);
    p.bar = reinterpret_cast<unsigned*>(pw + P.bar);
    p.status = reinterpret_cast<int*>(pw + P.status);
    p.abort_flag = reinterpret_cast<int*>(pw + P.abort_flag);
    if (c->mixed_max[k] == 0) continue;
    const Layout& L = c->Lm[k];
    unsigned char* w = c->ws + c->mbase[k];
    p.B = reinterpret_cast<float2*>(w + L.B);
    p.mT = reinterpret_cast<float*>(w + L.mT);
    p.partials = reinterpret_cast<double*>(w + L.partials);
    p.twx = reinterpret_cast<const float2*>(w + L.twx);
    p.twy = reinterpret_cast<const float2*>(w + L.twy);
    p.ones = reinterpret_cast<const float*>(w + L.ones);
    p.mask_flags = reinterpret_cast<int*>(w + L.mask_flags);
    p.energy = reinterpret_cast<const double*>(w + L.energy);
    if (batch[k] == 0) continue;
    p.I = target_intensity[k];
    p.phi_in = phase_in ? phase_in[k] : nullptr;
    p.phi_out = phase_out[k];
    p.r_out = residual_out ? residual_out[k] : nullptr;
    p.g_out = object_gap_out ? object_gap_out[k] : nullptr;
  }
  int it0 = 0;
  do {
    int it1 = it0 + gsk::kMaxIterPerLaunch;
    if (it1 > iters) it1 = iters;
    for (int k = 0; k < 3; ++k) {
      mp.cls[k].it0 = it0;
      mp.cls[k].it1 = it1;
      mp.cls[k].do_init = (it0 == 0) ? 1 : 0;
      mp.cls[k].do_final = (it1 == iters) ? 1 : 0;
    }
    // counter before every launch, abort word (next to it) before the first
    if (cudaMemsetAsync(mp.cls[0].bar, 0, (it0 == 0 ? 2 : 1) * sizeof(unsigned), c->stream) != cudaSuccess ||
        gsk::launch_mixed(mp, grid, c->tc_mode, c->stream) != cudaSuccess) {
      cudaGetLastError();
      return GS_ECUDA;
    }
    it0 = it1;
  } while (it0 < iters);
  return GS_OK;
}

int gs_status(gs_ctx* c) {
  if (c == nullptr) return GS_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  int st = 0;
  int* dst = at<int>(c, c->L.status);
  if (cudaMemcpyAsync(&st, dst, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemsetAsync(dst, 0, sizeof(int), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  return st;
}

int gs_run_host(gs_ctx* c, const float* target_intensity, const float* phase_in, int iters, float* phase_out,
                double* residual_out, double* object_gap_out) {
  const bool from_target = (c != nullptr) && (c->flags & GS_INIT_FROM_TARGET);
  if (c == nullptr || c->mixed || target_intensity == nullptr || (phase_in == nullptr && !from_target) ||
      phase_out == nullptr || iters < 0)
    return GS_EINVAL;
  const size_t n = static_cast<size_t>(c->nx) * c->ny;
  const size_t nres = static_cast<size_t>(iters) + 1;
  const size_t need = nres + static_cast<size_t>(iters);
  if (c->dres_cap < need) {
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
      cudaGetLastError();
      return GS_ECUDA;
    }
    cudaFree(c->dres);
    cudaFreeHost(c->hres);
    c->dres = nullptr;
    c->hres = nullptr;
    c->dres_cap = 0;
    if (cudaMalloc(&c->dres, need * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->hres, (need + 1) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return GS_ENOMEM;
    }
    c->dres_cap = need;
  }
  float* dI = at<float>(c, c->L.dI);
  float* dphi = at<float>(c, c->L.dphi);
  double* dr = residual_out ? c->dres : nullptr;
  double* dg = object_gap_out ? c->dres + nres : nullptr;
  if (cudaMemcpyAsync(dI, target_intensity, n * sizeof(float), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      (phase_in != nullptr &&
       cudaMemcpyAsync(dphi, phase_in, n * sizeof(float), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  int rc = gs_run(c, dI, dphi, iters, dphi, dr, dg);
  if (rc != GS_OK) return rc;
  // The phase goes straight to the caller's buffer; the gaps and the status
  // word go through the context's pinned staging, so that one synchronisation
  // ends the call whatever kind of host memory the caller passed.
  const size_t nr = static_cast<size_t>(iters) + ((c->flags & GS_FINAL_RESIDUAL) ? 1 : 0);
  int* dst = at<int>(c, c->L.status);
  int* hst = reinterpret_cast<int*>(c->hres + need);
  if (cudaMemcpyAsync(phase_out, dphi, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      ((dr || dg) &&
       cudaMemcpyAsync(c->hres, c->dres, need * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) ||
      cudaMemcpyAsync(hst, dst, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemsetAsync(dst, 0, sizeof(int), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  if (dr && nr) std::memcpy(residual_out, c->hres, nr * sizeof(double));
  if (dg && iters) std::memcpy(object_gap_out, c->hres + nres, static_cast<size_t>(iters) * sizeof(double));
  return *hst;
}

namespace {

struct AdamArgs {
  float* phase;
  float* m;
  float* v;
  int* state;
  float lr, beta1, beta2, eps;
  int steps;  // in this launch, 1 .. kMaxAdamStepsPerLaunch
};

int enqueue_loss(gs_ctx* c, const float* target_intensity, const float* phase, double* loss_out, float* grad_out,
                 double* phys_out, int mode = gsk::kLossFused, const AdamArgs* adam = nullptr) {
  gsk::LossParams p{};
  if (adam != nullptr) {
    p.phase = adam->phase;
    p.m = adam->m;
    p.v = adam->v;
    p.state = adam->state;
    p.lr = adam->lr;
    p.beta1 = adam->beta1;
    p.beta2 = adam->beta2;
    p.eps = adam->eps;
    p.steps = adam->steps;
  }
  p.mode = mode;
  // the fused and prepare launches stage their target over the previous one
  c->loss_prepared = (mode == gsk::kLossPrepare) || (mode == gsk::kLossStep && c->loss_prepared);
  p.n = c->nx;
  p.logn = ilog2i(c->nx);
  p.B = at<float2>(c, c->L.B);
  p.IT = at<float>(c, c->L.mT);
  p.I = target_intensity;
  p.phi = phase;
  p.grad = grad_out;
  p.loss = loss_out;
  p.phys = phys_out;
  p.p_slm = c->p_slm;
  p.energy = at<double>(c, c->L.energy);
  p.partials = at<double>(c, c->L.partials);
  p.tw = at<float2>(c, c->L.twx);
  p.bar = at<unsigned>(c, c->L.bar);
  p.status = at<int>(c, c->L.status);
  p.abort_flag = at<int>(c, c->L.abort_flag);
  p.inv_n = 1.0f / static_cast<float>(static_cast<double>(c->nx) * c->ny);
  if (cudaMemsetAsync(p.bar, 0, 2 * sizeof(unsigned), c->stream) != cudaSuccess ||  // counter and abort word
      gsk::launch_loss(p, choose_grid(c), c->stream) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  return GS_OK;
}

}  // namespace

int gs_loss_grad(gs_ctx* c, const float* target_intensity, const float* phase, double* loss_out, float* grad_out) {
  if (c == nullptr || c->mixed || target_intensity == nullptr || phase == nullptr || loss_out == nullptr ||
      c->nx != c->ny || gsk::uses_general(c->nx, c->ny))
    return GS_EINVAL;
  return enqueue_loss(c, target_intensity, phase, loss_out, grad_out, nullptr);
}

int gs_loss_prepare(gs_ctx* c, const float* target_intensity) {
  if (c == nullptr || c->mixed || target_intensity == nullptr || c->nx != c->ny || gsk::uses_general(c->nx, c->ny))
    return GS_EINVAL;
  return enqueue_loss(c, target_intensity, nullptr, nullptr, nullptr, nullptr, gsk::kLossPrepare);
}

int gs_loss_grad_prepared(gs_ctx* c, const float* phase, double* loss_out, float* grad_out) {
  if (c == nullptr || c->mixed || phase == nullptr || loss_out == nullptr || c->nx != c->ny ||
      gsk::uses_general(c->nx, c->ny) || !c->loss_prepared)
    return GS_EINVAL;
  return enqueue_loss(c, nullptr, phase, loss_out, grad_out, nullptr, gsk::kLossStep);
}

int gs_loss_adam_prepared(gs_ctx* c, float* phase, float* m, float* v, int* state, float lr, float beta1,
                          float beta2, float eps, double* loss_out) {
  if (c == nullptr || c->mixed || phase == nullptr || m == nullptr || v == nullptr || state == nullptr ||
      loss_out == nullptr || c->nx != c->ny || gsk::uses_general(c->nx, c->ny) || !c->loss_prepared ||
      !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return GS_EINVAL;
  const AdamArgs a{phase, m, v, state, lr, beta1, beta2, eps, 1};
  return enqueue_loss(c, nullptr, phase, loss_out, nullptr, nullptr, gsk::kLossStep, &a);
}

int gs_loss_adam_run(gs_ctx* c, float* phase, float* m, float* v, int* state, float lr, float beta1, float beta2,
                     float eps, int steps, double* loss_out) {
  if (c == nullptr || c->mixed || phase == nullptr || m == nullptr || v == nullptr || state == nullptr ||
      loss_out == nullptr || steps < 1 || c->nx != c->ny || gsk::uses_general(c->nx, c->ny) || !c->loss_prepared ||
      !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return GS_EINVAL;
  for (int k0 = 0; k0 < steps;) {  // launches of at most kMaxAdamStepsPerLaunch steps
    const int n = steps - k0 < gsk::kMaxAdamStepsPerLaunch ? steps - k0 : gsk::kMaxAdamStepsPerLaunch;
    const AdamArgs a{phase, m, v, state, lr, beta1, beta2, eps, n};
    const int rc = enqueue_loss(c, nullptr, phase, loss_out + k0, nullptr, nullptr, gsk::kLossStep, &a);
    if (rc != GS_OK) return rc;
    k0 += n;
  }
  return GS_OK;
}

int gs_physical_error(gs_ctx* c, const float* target_intensity, const float* phase, double* error_out) {
  if (c == nullptr || c->mixed || target_intensity == nullptr || phase == nullptr || error_out == nullptr ||
      c->nx != c->ny || gsk::uses_general(c->nx, c->ny))
    return GS_EINVAL;
  return enqueue_loss(c, target_intensity, phase, at<double>(c, c->L.lossbuf), nullptr, error_out);
}

int gs_set_slm_amplitude(gs_ctx* c, const float* amplitude) {
  if (c == nullptr || c->mixed) return GS_EINVAL;
  c->p_slm = amplitude;
  if (amplitude != nullptr &&
      gsk::launch_energy(amplitude, static_cast<long long>(c->nx) * c->ny, at<double>(c, c->L.energy), c->stream) !=
          cudaSuccess) {
    cudaGetLastError();
    c->p_slm = nullptr;
    return GS_ECUDA;
  }
  return GS_OK;
}

int gs_test_barrier_timeout(gs_ctx* c, int enable) {
  if (c == nullptr || enable < 0) return GS_EINVAL;
  c->extra_arrivals = enable ? 1u : 0u;
  return GS_OK;
}

int gs_check_workspace(gs_ctx* c) {
  if (c == nullptr) return GS_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  if (!c->mixed) return check_guards(c->ws, c->L);
  for (int k = 0; k < 3; ++k) {
    if (c->mixed_max[k] == 0) continue;
    const int rc = check_guards(c->ws + c->mbase[k], c->Lm[k]);
    if (rc != GS_OK) return rc;
  }
  return GS_OK;
}

int gs_test_corrupt_workspace(gs_ctx* c) {
  if (c == nullptr) return GS_EINVAL;
  const Layout& L = c->L;  // of a mixed context: its first class, at offset 0
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemset(c->ws + L.guard[0] + kGuardBytes / 2, 0, 1) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  return GS_OK;
}

int gs_set_trace(gs_ctx* c, int enable) {
  if (c == nullptr || enable < 0 || c->mixed) return GS_EINVAL;
  c->trace = enable != 0;
  return GS_OK;
}

int gs_get_trace(gs_ctx* c, unsigned long long* host_out, int capacity, int* passes, int* grid) {
  if (c == nullptr || host_out == nullptr || passes == nullptr || grid == nullptr || capacity < 0 || c->mixed)
    return GS_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  *passes = c->trace_passes;
  *grid = c->trace_grid;
  const long long need = 2LL * (c->trace_passes + 1) * c->trace_grid;
  if (need > capacity) return GS_EINVAL;
  if (need > 0 && cudaMemcpy(host_out, at<unsigned long long>(c, c->L.trace), need * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  return GS_OK;
}

int gs_set_mask_group(gs_ctx* c, int masks) {
  if (c == nullptr || masks < 0) return GS_EINVAL;
  c->group_override = masks;
  return GS_OK;
}

int gs_set_grid(gs_ctx* c, int ctas) {
  if (c == nullptr || ctas < 0) return GS_EINVAL;
  c->grid_override = ctas;
  return GS_OK;
}

int gs_get_grid(gs_ctx* c, int* ctas) {
  if (c == nullptr || ctas == nullptr) return GS_EINVAL;
  if (c->mixed) {
    int largest = 0;
    for (int k = 0; k < 3; ++k)
      if (c->mixed_max[k] > 0) largest = k;
    *ctas = choose_grid_for(c, static_cast<long long>(256 << largest) * (256 << largest));
    return GS_OK;
  }
  *ctas = choose_grid(c);
  return GS_OK;
}

int gs_destroy(gs_ctx* c) {
  if (c == nullptr) return GS_OK;
  int rc = GS_OK;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = GS_ECUDA;
  if (c->ws && cudaFree(c->ws) != cudaSuccess) rc = GS_ECUDA;
  if (c->dres && cudaFree(c->dres) != cudaSuccess) rc = GS_ECUDA;
  if (c->hres && cudaFreeHost(c->hres) != cudaSuccess) rc = GS_ECUDA;
  cudaGetLastError();
  delete c;
  return rc;
}

}  // extern "C"
