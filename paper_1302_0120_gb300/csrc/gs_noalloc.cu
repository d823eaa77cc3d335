// gs_noalloc.cu -- gs_run_noalloc: the iteration kernel with library-owned
// static scratch, for callers that must not allocate device memory.
//
// The scratch the iteration needs (field, amplitude, FP64 partial sums,
// twiddle tables, barrier and status words) lives in one file-scope
// __device__ array of fixed size; every GPU that loads the library holds it
// until the process exits. The array's name is only a host-side stand-in in
// host code, so its device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels. This file calls no
// cudaMalloc, cudaFree or other allocating routine.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "gs.h"
#include "gs_fft.cuh"
#include "gs_internal.h"

namespace {

constexpr int kMaxPixels = 512 * 512;    // largest nx * ny served from the static scratch
constexpr int kMaxGrid = 256;            // blocks per launch (partial-sum rows)
constexpr int kTwEntries = 31 * 32 + 31 * 1024;  // one stage-twiddle table (see gs_fft.cuh)
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

constexpr size_t kOffB = 0;
constexpr size_t kOffM = align_up(kOffB + static_cast<size_t>(kMaxPixels) * 8);
constexpr size_t kOffPartials = align_up(kOffM + static_cast<size_t>(kMaxPixels) * 4);
constexpr size_t kOffTwx = align_up(kOffPartials + static_cast<size_t>(gsk::kSlots) * kMaxGrid * 8);
constexpr size_t kOffTwy = align_up(kOffTwx + static_cast<size_t>(kTwEntries) * 8);
constexpr size_t kOffOnes = align_up(kOffTwy + static_cast<size_t>(kTwEntries) * 8);
constexpr size_t kOffWords = align_up(kOffOnes + 4096 * sizeof(float));
constexpr size_t kScratchBytes = align_up(kOffWords + (3 + gsk::kMaxBatch) * sizeof(int));  // barrier, status, abort, mask flags

// The shared scratch of every gs_run_noalloc call on this device (about 4 MiB).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceScratch {
  unsigned char* base = nullptr;  // device address of g_scratch on that device
  int num_sms = 0;
};
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

bool valid_dim(int n) { return n >= 32 && n <= 4096 && (n & (n - 1)) == 0; }

int log2_exact(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Stage twiddle tables of a length-n transform, the same layout and values
// (double precision rounded once, exact octant points) as the context path.
__global__ void twiddle_tables(float2* tw, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kTwEntries; e += gridDim.x * blockDim.x) {
    const int nsl = e < 31 * 32 ? 5 : 10;
    const int off = gsk::twiddle_offset(nsl);
    const int ns = 1 << nsl;
    float2 w = make_float2(0.f, 0.f);
    if (n > ns) {
      const int R = (n / ns > 32) ? 32 : n / ns;
      const int m = (e - off) / ns + 1;
      const int r = (e - off) % ns;
      if (m < R) {
        const long long M = static_cast<long long>(ns) * R;
        const long long k = (static_cast<long long>(r) * m) % M;
        if ((8 * k) % M == 0) {
          const double h = 0.70710678118654752440;
          const double oc[8] = {1.0, h, 0.0, -h, -1.0, -h, 0.0, h};
          const double os[8] = {0.0, h, 1.0, h, 0.0, -h, -1.0, -h};
          const int o = static_cast<int>((8 * k) / M);
          w = make_float2(static_cast<float>(oc[o]), static_cast<float>(-os[o]));
        } else {
          double s, c;
          sincospi(2.0 * static_cast<double>(k) / static_cast<double>(M), &s, &c);
          w = make_float2(static_cast<float>(c), static_cast<float>(-s));
        }
      }
    }
    tw[e] = w;
  }
}

__global__ void fill_ones(float* x, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) x[e] = 1.0f;
}

// Device address of the static scratch on the current device; looked up on
// the first call for that device.
int scratch_for_current_device(unsigned char** base, int* num_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceScratch& d = g_dev[dev];
  if (d.base == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr ||
        cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return GS_ECUDA;
    }
    d.base = static_cast<unsigned char*>(p);
  }
  *base = d.base;
  *num_sms = d.num_sms;
  return GS_OK;
}

}  // namespace

extern "C" int gs_run_noalloc(int nx, int ny, unsigned flags, void* stream, const float* target_intensity,
                              const float* phase_in, int iters, float* phase_out, double* residual_out,
                              double* object_gap_out, int* device_status) {
  if (!valid_dim(nx) || !valid_dim(ny) || static_cast<long long>(nx) * ny > kMaxPixels) return GS_EINVAL;
  if ((flags & ~static_cast<unsigned>(GS_FINAL_RESIDUAL | GS_INIT_FROM_TARGET)) != 0) return GS_EINVAL;
  const bool from_target = (flags & GS_INIT_FROM_TARGET) != 0;
  if (target_intensity == nullptr || (phase_in == nullptr && !from_target) || phase_out == nullptr || iters < 0)
    return GS_EINVAL;
  unsigned char* base = nullptr;
  int num_sms = 0;
  int rc = scratch_for_current_device(&base, &num_sms);
  if (rc != GS_OK) return rc;
  int per_sm = 0;
  if (gsk::iteration_occupancy(nx, ny, &per_sm) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  // the context path's rule: one block per 4096 pixels, and small grids up
  // to 32 blocks (one per 2048 pixels)
  const long long npx = static_cast<long long>(nx) * ny;
  int grid = static_cast<int>(npx / 4096);
  const int small = static_cast<int>(npx / 2048 < 32 ? npx / 2048 : 32);
  if (grid < small) grid = small;
  if (grid > num_sms * per_sm) grid = num_sms * per_sm;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) grid = 1;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gsk::Params p{};
  p.nx = nx;
  p.ny = ny;
  p.lognx = log2_exact(nx);
  p.logny = log2_exact(ny);
  p.B = reinterpret_cast<float2*>(base + kOffB);
  p.mT = reinterpret_cast<float*>(base + kOffM);
  p.I = target_intensity;
  p.phi_in = phase_in;
  p.phi_out = phase_out;
  p.partials = reinterpret_cast<double*>(base + kOffPartials);
  p.r_out = residual_out;
  p.g_out = object_gap_out;
  p.twx = reinterpret_cast<float2*>(base + kOffTwx);
  p.twy = reinterpret_cast<float2*>(base + kOffTwy);
  p.bar = reinterpret_cast<unsigned*>(base + kOffWords);
  p.status = reinterpret_cast<int*>(base + kOffWords) + 1;
  p.abort_flag = reinterpret_cast<int*>(base + kOffWords) + 2;
  p.mask_flags = reinterpret_cast<int*>(base + kOffWords) + 3;
  p.ones = reinterpret_cast<const float*>(base + kOffOnes);
  p.batch = 1;
  p.group = 1;
  p.init_target = from_target ? 1 : 0;
  p.mstride = static_cast<long long>(nx) * ny;
  p.rstride = iters + ((flags & GS_FINAL_RESIDUAL) ? 1 : 0);
  p.gstride = iters;
  p.iters = iters;
  p.final_resid = (flags & GS_FINAL_RESIDUAL) ? 1 : 0;
  p.extra_arrivals = 0;
  const double n = static_cast<double>(nx) * ny;
  p.inv_sqrt_n = static_cast<float>(1.0 / std::sqrt(n));
  p.inv_n = 1.0 / n;

  // The scratch keeps the previous call's contents: clear the words that must
  // start at zero and rebuild the twiddle tables for this size.
  if (cudaMemsetAsync(base + kOffWords, 0, 3 * sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  fill_ones<<<16, 256, 0, s>>>(reinterpret_cast<float*>(base + kOffOnes), 4096);
  twiddle_tables<<<64, 256, 0, s>>>(const_cast<float2*>(p.twx), nx);
  twiddle_tables<<<64, 256, 0, s>>>(const_cast<float2*>(p.twy), ny);
  if (cudaGetLastError() != cudaSuccess) return GS_ECUDA;
  int it0 = 0;
  do {
    int it1 = it0 + gsk::kMaxIterPerLaunch;
    if (it1 > iters) it1 = iters;
    p.it0 = it0;
    p.it1 = it1;
    p.do_init = (it0 == 0) ? 1 : 0;
    p.do_final = (it1 == iters) ? 1 : 0;
    if (cudaMemsetAsync(p.bar, 0, sizeof(unsigned), s) != cudaSuccess ||
        gsk::launch_iterations(p, grid, s) != cudaSuccess) {
      cudaGetLastError();
      return GS_ECUDA;
    }
    it0 = it1;
  } while (it0 < iters);
  if (device_status != nullptr &&
      cudaMemcpyAsync(device_status, p.status, sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  return GS_OK;
}
