// gs_internal.h -- parameters shared by the host API and the iteration kernel.
#pragma once

#include <cuda_runtime.h>

namespace gsk {

constexpr int kThreads = 256;                   // threads per block of the iteration kernel
constexpr int kMaxIterPerLaunch = 128;          // iterations per persistent launch
constexpr int kSlots = 2 * kMaxIterPerLaunch + 2;  // FP64 partial-sum slots per launch
constexpr int kMaxGrid = 256;                   // upper bound on blocks per launch
constexpr int kMaxBatch = 64;                   // masks per launch
// Pass timestamps (gs_set_trace): rows of kMaxGrid (done, released) pairs,
// row 0 the launch start, row 1 + q pass q of the launch.
constexpr int kTraceRows = 2 * kMaxIterPerLaunch + 4;
// Group exchange buffers: (256 / T) groups of (n + n/32) complex, T = n/32,
// which is 256 * 33 complex whatever n is.
constexpr int kGroupSmemBytes = kThreads * 33 * 8;
// Extra shared memory of the tensor-core kernels: stage twiddles [32][32]
// complex and a 32-entry cos/sin table (mma.sync); the two DFT matrices (hi
// and lo parts, 8 KiB each) and an 8 KiB twiddle table (tcgen05, whose
// operands share the exchange buffers).
constexpr int kTcExtraSmemBytes = 32 * 32 * 8 + 32 * 8;
constexpr int kTc5ExtraSmemBytes = 4 * 64 * 64 * 2 + 32 * 32 * 8;
// The mixed launch on tcgen05: the 32-point matrix (hi, lo), the 8-, 16- and
// 32-point matrices (hi, lo) and three twiddle tables.
constexpr int kMixedTc5ExtraSmemBytes = 2 * 64 * 64 * 2 + 2 * (16 * 16 + 32 * 32 + 64 * 64) * 2 + 3 * 32 * 32 * 8;

struct Params {
  int nx, ny;          // grid, powers of two in [32, 4096]
  int lognx, logny;
  float2* B;           // [ny][nx] field between passes (row-transformed)
  float* mT;           // scaled OSP amplitude, transposed: [nx][ny]
  const float* I;      // target intensity [ny][nx]
  const float* phi_in; // initial phase [ny][nx]
  float* phi_out;      // final phase [ny][nx]
  double* partials;    // [kSlots][batch][grid] per-block FP64 sums
  double* r_out;       // r^nu, or null
  double* g_out;       // g^nu, or null
  const float2* twx;   // stage twiddle tables of the row transforms (length nx)
  const float2* twy;   // stage twiddle tables of the column transforms (length ny)
  unsigned* bar;       // grid barrier arrival counter (zeroed before each launch)
  int* status;         // device status word (first error wins)
  int* abort_flag;     // set when a launch failed; later launches of the run return at once
  int* mask_flags;     // [kMaxBatch]: 1 for a mask whose target was rejected (written by the first launch)
  int batch;           // masks in this launch, 1..kMaxBatch, strided in every array
  long long mstride;   // elements of one mask in I, phi_in, phi_out, B and mT (nx*ny)
  int rstride;         // entries of one mask in r_out
  int gstride;         // entries of one mask in g_out
  int it0, it1;        // iterations [it0, it1) of this launch
  int iters;           // total K of the run
  int do_init;         // this launch computes m and u^0
  int do_final;        // this launch ends the run (phase out, final residual)
  int final_resid;     // compute r^K
  const float* p_slm;  // SLM amplitude p [ny][nx] (Eq. slm-constraint), or null for p = 1
  const double* energy;  // sum p^2 (FP64, workspace) when p_slm is set
  const float* ones;   // a row of max(nx, ny) ones (workspace): p when p_slm is null
  int init_target;     // start from P_S(F^{-1} m) instead of p exp(i phi_in)
  unsigned extra_arrivals;  // test hook: arrivals a barrier waits for beyond the grid (0 in use)
  float inv_sqrt_n;    // 1/sqrt(N)
  double inv_n;        // 1/N
  int tensor_core;     // host side: transforms on the FP32 ALUs (0) or the tensor cores (square 256,
                       // 512, 1024): mma.sync (1), tcgen05 with FP16 (2) or BF16 (3) operands
  unsigned long long* trace;  // [kTraceRows][grid][2] globaltimer stamps of block 0's thread 0 per block, or null
  int group;           // masks iterated together, 1..batch: the batch runs group after group
                       // through the whole schedule, so that a group's fields stay in L2
  // Grids with a side that is not a power of two (gs_general.cuh): the
  // radices of the row and column transforms, 3 bits per stage (code c means
  // radix kRadixOf[c]), first stage in the low bits, and the stage counts.
  unsigned planx, plany;
  int nstx, nsty;
};

// Three size classes in one launch: square grids 256, 512 and 1024
// (log2 n = 8 + c), any of them with an empty batch. Every class has the
// same iteration count, flags and chunk; the barrier, status and abort words
// are class 0's. Mask flags and partial sums are per class.
struct MixedParams {
  Params cls[3];
};

// Small grids (power-of-two sides >= 32, at most this many pixels) run one
// block per mask with the whole field in shared memory (gs_small.cuh).
constexpr int kSmallMaxPixels = 8192;
inline __host__ __device__ bool small_grid(int nx, int ny) {
  const bool px = nx > 0 && (nx & (nx - 1)) == 0, py = ny > 0 && (ny & (ny - 1)) == 0;
  return px && py && nx >= 32 && ny >= 32 && static_cast<long long>(nx) * ny <= kSmallMaxPixels;
}

// The general kernel serves every grid with a side that is not a power of
// two or is below 32 (the power-of-two kernels need 32 points per thread).
inline __host__ __device__ bool uses_general(int nx, int ny) {
  const bool px = nx > 0 && (nx & (nx - 1)) == 0, py = ny > 0 && (ny & (ny - 1)) == 0;
  return !px || !py || nx < 32 || ny < 32;
}

// Register-resident general-grid kernel (gs_rg.cuh): sides n = T V with a
// line in one warp (T lanes of V points, T, V <= 32). rg_threads(n) is T for
// the sides it serves (600 = 24 x 25, 768 = 32 x 24, 800 = 32 x 25,
// 1024 = 32 x 32), else 0; a grid whose two sides are both served, and not
// both powers of two, runs there (800 x 600, 1024 x 768, ...); any other grid
// with a side that is not a power of two on the shared-memory general kernel.
// Kernel templates take such a side itself in place of log2 nx (is_rg_side).
inline __host__ __device__ constexpr int rg_threads(int n) {
  return n == 600 ? 24 : (n == 768 || n == 800 || n == 1024) ? 32 : 0;
}
inline __host__ __device__ constexpr bool is_rg_side(int lx) { return lx >= 32; }
inline __host__ __device__ bool uses_rg(int nx, int ny) {
  return rg_threads(nx) > 0 && rg_threads(ny) > 0 && !(nx == 1024 && ny == 1024);
}

// Sides of the general kernel: 5-smooth (2^a 3^b 5^c) in [8, kMaxGeneralSide].
constexpr int kMaxGeneralSide = 1536;
constexpr int kMaxGeneralStages = 10;

// The general kernel transforms a row or column with a team of two warps;
// a block holds four teams.
constexpr int kGenTeam = 64;
constexpr int kGenTeams = kThreads / kGenTeam;

// Shared-memory layout of the general kernel: the two twiddle tables (nx,
// then ny complex), then per team two buffers of max(nx, ny) complex.
inline __host__ __device__ int gen_tw_entries(int nx, int ny) { return (nx + ny + 1) & ~1; }
inline __host__ __device__ int gen_team_stride(int nmax) { return 2 * nmax + 2; }  // complex; 16-byte multiple
inline __host__ __device__ size_t gen_smem_bytes(int nx, int ny) {
  const int nmax = nx > ny ? nx : ny;
  return (static_cast<size_t>(gen_tw_entries(nx, ny)) + static_cast<size_t>(kGenTeams) * gen_team_stride(nmax)) *
         sizeof(float2);
}

// Kernel for log2(nx) = LX and the given log2(ny); defined per LX in gs_inst.cu.
template <int LX>
const void* iterate_kernel_lx(int ly);
// Kernel with tensor-core transforms for an n x n grid, log2(n) = l in 8..10
// (gs_tc_inst.cu); null otherwise.
const void* iterate_kernel_tc(int l);
// Kernel for grids with a side that is not a power of two (gs_general_inst.cu).
const void* iterate_kernel_general();
// Register-resident kernel for an nx x ny grid with uses_rg (gs_rg_inst.cu),
// its dynamic shared memory, and the layout of its twiddle tables: for a side
// n = T V, n entries W_n^{t q} at [q T + t] (q < V, t < T), then n entries
// W_n^{q j} at [j V + q].
const void* iterate_kernel_rg(int nx, int ny);
size_t rg_smem_bytes(int nx, int ny);
// The kernels and shared memory for one row length, from the object of
// gs_rg_inst.cu compiled for it.
template <int NX>
const void* iterate_kernel_rg_nx(int ny);
template <int NX>
size_t rg_smem_bytes_nx(int ny);
// Stage twiddle tables of a power-of-two length n (the layout stage_c reads),
// kStageTwiddleEntries entries, rounded once from double (gs_api.cu).
constexpr int kStageTwiddleEntries = 31 * 32 + 31 * 1024;
void stage_twiddles_host(int n, float2* out);
// Kernel for three square size classes in one launch (gs_mixed_inst.cu), by
// TcMode.
const void* iterate_kernel_mixed(int tc_mode);
size_t mixed_smem_bytes(int tc_mode);
cudaError_t mixed_occupancy(int tc_mode, int* blocks_per_sm);
cudaError_t launch_mixed(const MixedParams& mp, int grid, int tc_mode, cudaStream_t s);

// Tensor-core modes of Params::tensor_core.
enum TcMode { kTcNone = 0, kTcMmaSync = 1, kTcGen05F16 = 2, kTcGen05Bf16 = 3 };
size_t iteration_smem_bytes(int nx, int ny, int tc_mode = kTcNone);

// Intensity loss and gradient (square grids), see gs_loss.cuh. A launch
// either does everything (fused), or stages the target once (prepare) for
// later launches that run only the transform passes on it (step).
enum LossMode { kLossFused = 0, kLossPrepare = 1, kLossStep = 2 };
struct LossParams {
  int n, logn;             // square grid n x n
  float2* B;               // workspace field (column-blocked layout)
  float* IT;               // workspace: target transposed [n][n]
  const float* I;          // target intensity [n][n]
  const float* phi;        // phase [n][n]
  float* grad;             // dL/dphi [n][n], or null (loss only)
  double* loss;            // [steps]: the loss before each step
  double* phys;            // [2]: physical error (E_l, E_d), or null
  const float* p_slm;      // SLM amplitude [n][n], or null (p = 1)
  const double* energy;    // sum p^2 when p_slm is set
  double* partials;        // [6][grid]
  const float2* tw;        // stage twiddle tables (length n)
  unsigned* bar;
  int* status;
  int* abort_flag;
  float inv_n;             // 1/N
  int mode;                // LossMode: fused, prepare the target, or a step on the prepared target
  // A step with the Adam update fused into the gradient pass (grad is then
  // null): phase (the same array as phi) is updated in place with the running
  // moments m, v; state[0] counts the steps done, state[1] the blocks done.
  float* phase;
  float* m;
  float* v;
  int* state;
  float lr, beta1, beta2, eps;
  // Adam steps in this launch (1 unless m is set): the gradient pass of a
  // step also forms the next step's row transforms of exp(i phase).
  int steps;
};

// Adam steps per launch of gs_loss_adam_run (a longer run is split).
constexpr int kMaxAdamStepsPerLaunch = 1024;

cudaError_t launch_loss(const LossParams& p, int grid, cudaStream_t s);
cudaError_t launch_iterations(const Params& p, int grid, cudaStream_t s);
// sum p^2 of an SLM amplitude into *energy (NaN if p has a negative or non-finite value)
cudaError_t launch_energy(const float* p, long long n, double* energy, cudaStream_t s);
cudaError_t iteration_occupancy(int nx, int ny, int* blocks_per_sm, int tc_mode = kTcNone);
// The tcgen05 kernel of n x n masks, log2(n) = l in 8..10 (gs_tc5_inst.cu);
// FP16 or BF16 operands; null for other sizes.
const void* iterate_kernel_tc5(int l, bool bf16);
// Small grids (small_grid): allow the kernel its shared memory, and launch
// one block per mask of p.batch (gs_small_inst.cu).
cudaError_t small_prepare(int nx, int ny);
cudaError_t launch_small(const Params& p, cudaStream_t s);

}  // namespace gsk
