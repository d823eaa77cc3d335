/*
 * gs.h -- C ABI of the GB300 Gerchberg-Saxton phase-mask library.
 *
 * The library computes a phase-only mask for a spatial light modulator (SLM)
 * whose Fourier-transform intensity reproduces a target optical stimulation
 * pattern (OSP), by the method of alternating projections (Gerchberg-Saxton)
 * of Kramer, Hagemann and Luke, "Real-Time Phase Masks for Interactive
 * Stimulation of Optogenetic Neurons", Sec. II:
 *
 *   S = { u : |u_jk| = 1 }                 (Eq. slm-constraint, unit amplitude p = 1)
 *   M = { u : |(F u)_jk| = m_jk }          (Eq. pattern-constraint)
 *   u^{nu+1} = P_S P_M u^nu                (Eq. e:AP, projections Eqs. e:PS, e:PM, e:Mhat)
 *
 * Conventions shared by every entry point:
 *   - A grid is nx x ny pixels stored row-major as [ny][nx] (pixel (j, k) of
 *     the paper, j < nx along a row, at index k*nx + j: the paper's
 *     lexicographic pixel index, Sec. III).
 *   - F is the 2D DFT with kernel exp(-2 pi i (j k1/nx + k k2/ny)). The target
 *     intensity I is given in DFT order (zero frequency at [0][0]).
 *   - The OSP amplitude is m = sqrt(I) scaled so that sum m^2 = N = nx*ny
 *     (m is an amplitude, Eq. pattern-constraint; the scale, which the paper
 *     leaves open, does not change the iterates).
 *   - A pixel whose value is exactly zero gets phase 0 in either projection
 *     (the paper allows any phase there, Eqs. e:PS and e:Mhat).
 *   - Residuals are the normalised gaps of Eq. (gap-error):
 *       r^nu = || |F u^nu|/sqrt(N) - m ||_2 / sqrt(N)   (distance of u^nu to M)
 *       g^nu = || P_M u^nu - P_S P_M u^nu ||_2 / sqrt(N) (distance of P_M u^nu to S)
 *     reduced in FP64. The field itself is computed in FP32.
 *   - nx and ny are powers of two in [8, 4096] or 5-smooth numbers
 *     (2^a 3^b 5^c, such as the 800 x 600 SLM of Sec. V) in [8, 1536].
 *     Grids with both sides powers of two of at least 32 run on the
 *     register-resident kernels (one block per mask when the grid has at
 *     most 8192 pixels, see gs_run); every other grid on the general kernel.
 *
 * Memory and ordering:
 *   - Pointers named "device" are CUDA device pointers owned by the caller;
 *     the library never frees them. Pointers named "host" are host memory
 *     owned by the caller (pinned memory gives asynchronous copies).
 *   - All work is enqueued on the context's CUDA stream and is asynchronous
 *     unless stated otherwise. Results are valid once that stream has
 *     synchronised (e.g. through gs_status).
 *   - A context is not thread-safe; use one context per host thread.
 *
 * Errors: every call returns an int status, GS_OK on success. No exception
 * crosses the ABI. Arguments are validated before anything is enqueued.
 * Errors detected on the device (a non-finite or all-zero target, a barrier
 * that timed out) are recorded in the context and returned by gs_status.
 */
#ifndef GS_GB300_H
#define GS_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GS_OK = 0,
  GS_EINVAL = -1,   /* invalid argument: null pointer, unsupported size, iters < 0 */
  GS_ENOMEM = -2,   /* device or host allocation failed */
  GS_ECUDA = -3,    /* a CUDA runtime call failed (no device, launch failure) */
  GS_ETIMEOUT = -4, /* a device-side wait gave up (grid barrier did not complete) */
  GS_ENUMERIC = -5, /* target intensity is non-finite, negative or sums to zero */
  GS_ECORRUPT = -6  /* gs_check_workspace: a canary word of the workspace was overwritten */
};

/* Flags for gs_create. */
enum {
  /* After the last iteration also compute r^K (one forward column pass). */
  GS_FINAL_RESIDUAL = 1u,
  /* Start from the target instead of an initial phase: u^0 = P_S(F^{-1} m),
   * the initial condition of Sec. IV (P_M uhat^0 of the paper, garbled in
   * the text, read this way). phase_in is ignored and may be NULL. With a
   * real target this start is conjugate-symmetric, so F u stays real. */
  GS_INIT_FROM_TARGET = 2u,
  /* Run the DFTs of Eq. (e:PM) and the inverse transforms on the tensor
   * cores: each length-n transform (n = 256, 512, 1024; square grids only) is
   * the four-step factorisation n = 32 x (n/32) with both stages as dense
   * DFT-matrix products, FP16 operands and FP32 accumulation; projections,
   * gaps and reductions are unchanged (FP32 field, FP64 sums). The paper
   * computes in single or double precision only (Sec. V); this reduced
   * precision form has no counterpart there. One iteration differs from the
   * FP32 one by about 1e-3 (relative L2). The operands are kept in the FP16
   * range by a power-of-two scale per mask (inputs below 2^15 from the bound
   * sqrt(n sum p^2) of every transform input; the scale is undone in FP32),
   * so any laser amplitude is accepted. The products run on the
   * fifth-generation tensor cores (tcgen05: operands in shared memory, FP32
   * accumulators in tensor memory, each stage M = 128 products over the rows
   * of four warps' lines). */
  GS_TENSOR_CORE = 4u,
  /* With GS_TENSOR_CORE: BF16 operands instead of FP16 (8 bits of
   * significand instead of 11, FP32's range), each split into its BF16
   * rounding and the rounding of the remainder, three products per K step,
   * to keep the FP16 form's accuracy. Not accepted without GS_TENSOR_CORE or
   * with GS_TC_MMA_SYNC. */
  GS_BF16 = 8u,
  /* With GS_TENSOR_CORE: run the products as warp-level mma.sync tiles (FP16)
   * instead of tcgen05, for comparison. Not accepted without GS_TENSOR_CORE
   * or with GS_BF16. */
  GS_TC_MMA_SYNC = 16u
};

typedef struct gs_ctx gs_ctx;

/*
 * gs_create -- allocate a context for nx x ny grids.
 *
 * Operation: none yet; sizes the workspace for Eq. (e:AP) on an nx x ny SLM
 * (Sec. II: "n_x, n_y the respective number of pixels").
 *   out     host pointer that receives the context (set to NULL on failure).
 *   nx, ny  grid sides: powers of two in [8, 4096], or 5-smooth in [8, 1536].
 *   flags   GS_* flags (GS_FINAL_RESIDUAL, GS_INIT_FROM_TARGET,
 *           GS_TENSOR_CORE, GS_BF16, GS_TC_MMA_SYNC).
 *   stream  a cudaStream_t, or NULL for the legacy default stream. All later
 *           work of this context is enqueued on it.
 * The context owns its device workspace (gs_workspace_bytes bytes): the field,
 * the scaled amplitude, per-block FP64 partial sums, twiddle tables, a
 * barrier counter and a status word. Synchronous (allocates and uploads).
 * Returns GS_EINVAL for bad sizes, an unknown flag, GS_TENSOR_CORE with a grid
 * other than 256, 512 or 1024 square, GS_BF16 or GS_TC_MMA_SYNC where they do
 * not apply, or a NULL out; GS_ENOMEM, GS_ECUDA.
 */
int gs_create(gs_ctx** out, int nx, int ny, unsigned flags, void* stream);

/*
 * gs_create_batched -- gs_create for up to max_batch masks per run.
 *
 * Same as gs_create; the workspace holds max_batch fields (1 <= max_batch
 * <= 64) so that gs_run_batched can iterate that many independent masks of
 * the same grid in one launch (Eq. e:AP for each). Returns GS_EINVAL for a
 * bad size or max_batch, GS_ENOMEM, GS_ECUDA.
 */
int gs_create_batched(gs_ctx** out, int nx, int ny, int max_batch, unsigned flags, void* stream);

/*
 * gs_run -- run K iterations of the method of alternating projections.
 *
 * Operation: Eq. (e:AP) from u^0 = exp(i phase_in), with P_S (Eq. e:PS, p = 1)
 * and P_M (Eqs. e:PM, e:Mhat, m from target_intensity); outputs the phase of
 * u^K and the gaps of Eq. (gap-error).
 *   target_intensity  device, float [ny][nx], DFT order, >= 0, finite, not all 0.
 *   phase_in          device, float [ny][nx], radians. May alias phase_out
 *                     (warm start from a previous mask). Ignored (may be
 *                     NULL) with GS_INIT_FROM_TARGET.
 *   iters             K >= 0. K == 0 computes r^0 only (with GS_FINAL_RESIDUAL)
 *                     and writes phase_out = arg exp(i phase_in).
 *   phase_out         device, float [ny][nx], arg u^K in (-pi, pi].
 *   residual_out      device, double[K+1] (r^0..r^K) with GS_FINAL_RESIDUAL,
 *                     else double[K] (r^0..r^{K-1}); or NULL.
 *   object_gap_out    device, double[K] (g^0..g^{K-1}), or NULL.
 * Asynchronous on the context stream. Returns GS_EINVAL on NULL context or
 * arrays, iters < 0; GS_ECUDA if a launch fails. Device-side errors are
 * reported by gs_status; on GS_ENUMERIC the phase output is left untouched and
 * residuals are set to NaN.
 * Execution: one persistent cooperative launch per 128 iterations; grids of
 * power-of-two sides >= 32 with at most 8192 pixels (64 x 64, 32 x 256, ...)
 * instead run the whole run in one launch of one block per mask with the
 * field in shared memory (same iterates bit for bit), unless gs_set_grid
 * fixed a grid, or the target start, a laser amplitude or pass timestamps
 * are in use.
 */
int gs_run(gs_ctx* c, const float* target_intensity, const float* phase_in, int iters,
           float* phase_out, double* residual_out, double* object_gap_out);

/*
 * gs_run_batched -- gs_run for `batch` independent masks of the same grid.
 *
 * Operation: Eq. (e:AP) for each mask b < batch, exactly as gs_run (the
 * masks share only the launch: phases are identical to separate runs; the
 * gaps agree to FP64 rounding, their partial sums being grouped by the
 * blocks' shares of the whole batch).
 * Every array is strided by mask, mask b at offset b * (per-mask size):
 *   target_intensity, phase_in, phase_out  device, float [batch][ny][nx]
 *   residual_out   device, double [batch][K+1] (GS_FINAL_RESIDUAL) or
 *                  [batch][K], or NULL
 *   object_gap_out device, double [batch][K], or NULL
 * 1 <= batch <= the context's max_batch. A mask whose target is invalid is
 * skipped (its phase untouched, its gaps NaN) and gs_status reports
 * GS_ENUMERIC; the other masks complete. Asynchronous; errors as gs_run.
 */
int gs_run_batched(gs_ctx* c, int batch, const float* target_intensity, const float* phase_in, int iters,
                   float* phase_out, double* residual_out, double* object_gap_out);

/*
 * gs_create_mixed -- a context for batches of square masks of three sizes,
 * 256 x 256, 512 x 512 and 1024 x 1024, iterated together in one launch.
 *
 * Operation: none yet; sizes one workspace per size (as gs_create_batched
 * for n = 256 << k with max_batch[k] masks) for gs_run_mixed, which runs
 * Eq. (e:AP) on every mask of every size in one persistent launch.
 *   out        host pointer that receives the context (NULL on failure).
 *   max_batch  host int[3]: masks of size 256 << k, each 0..64, sum 1..64.
 *   flags      GS_FINAL_RESIDUAL, GS_INIT_FROM_TARGET, GS_TENSOR_CORE (tcgen05
 *              products at every size), GS_BF16, GS_TC_MMA_SYNC.
 *   stream     a cudaStream_t, or NULL for the legacy default stream.
 * Only gs_run_mixed, gs_status, gs_set_grid, gs_get_grid and gs_destroy
 * accept a mixed context; the single-size calls return GS_EINVAL.
 * Returns GS_EINVAL for NULL pointers, a bad max_batch or an unknown flag;
 * GS_ENOMEM, GS_ECUDA.
 */
int gs_create_mixed(gs_ctx** out, const int* max_batch, unsigned flags, void* stream);

/*
 * gs_run_mixed -- enqueue K iterations of Eq. (e:AP) for batch[k] masks of
 * size n_k = 256 << k (k = 0, 1, 2) in one persistent launch (chunks of 128
 * iterations, as gs_run).
 *
 * Every pass of the launch visits the masks of all three sizes before its
 * grid barrier; each mask follows exactly the single-size path (same
 * transforms, projections and gaps), so its phase is bit-identical to a
 * gs_run_batched run of its size; its gaps can differ in the last bits
 * because the FP64 partial sums are grouped by the launch's block count.
 *   batch            host int[3], 0 <= batch[k] <= max_batch[k], sum >= 1.
 *   target_intensity host array of 3 device pointers; entry k: float
 *                    [batch[k]][n_k][n_k] (ignored when batch[k] = 0).
 *   phase_in         host array of 3 device pointers as above, or NULL
 *                    (whole array or entries) with GS_INIT_FROM_TARGET.
 *   iters            K >= 0.
 *   phase_out        host array of 3 device pointers, float
 *                    [batch[k]][n_k][n_k], may alias phase_in.
 *   residual_out     NULL or host array of 3 device pointers (entries may be
 *                    NULL): double [batch[k]][K (+1 with GS_FINAL_RESIDUAL)].
 *   object_gap_out   NULL or host array of 3 device pointers: double
 *                    [batch[k]][K].
 * Asynchronous on the context's stream; errors found on the device
 * (GS_ENUMERIC per mask, GS_ETIMEOUT) are reported by gs_status. Returns
 * GS_EINVAL for a NULL or non-mixed context, a bad batch, missing pointers or
 * K < 0; GS_ECUDA if a launch fails.
 */
int gs_run_mixed(gs_ctx* c, const int* batch, const float* const* target_intensity, const float* const* phase_in,
                 int iters, float* const* phase_out, double* const* residual_out, double* const* object_gap_out);

/*
 * gs_run_host -- gs_run on HOST buffers: end-to-end call including transfers.
 *
 * Same operation and argument meaning as gs_run, but every array is host
 * memory (pinned memory gives asynchronous copies): the target and the
 * initial phase are copied to context-owned device buffers, the iteration
 * runs, and the phase and residuals are copied back. Synchronous: returns
 * after the results are in host memory, with the device status folded into
 * the return value (GS_ENUMERIC, GS_ETIMEOUT as for gs_status).
 */
int gs_run_host(gs_ctx* c, const float* target_intensity, const float* phase_in, int iters,
                float* phase_out, double* residual_out, double* object_gap_out);

/*
 * gs_status -- wait for the context stream and return the device status.
 *
 * Synchronises the context stream, then returns GS_OK, GS_ENUMERIC or
 * GS_ETIMEOUT for the runs enqueued since the previous gs_status (the first
 * error wins), or GS_ECUDA if the stream reports an error. Clears the status.
 */
int gs_status(gs_ctx* c);

/*
 * gs_set_slm_amplitude -- the laser amplitude p on the SLM for later runs.
 *
 * Operation: replaces the unit amplitude of the SLM set S by p, Eq.
 * (slm-constraint): runs start from u^0 = p exp(i phase_in), P_S maps v to
 * p v/|v| (Eq. e:PS), the target amplitude carries the energy sum p^2, and
 * both gaps are divided by ||p||_2 instead of sqrt(N).
 *   amplitude  device, float [ny][nx], >= 0 and finite, caller-owned: it must
 *              stay valid while runs that use it execute. NULL restores p = 1.
 * Enqueues an FP64 reduction of sum p^2 on the context stream (asynchronous).
 * A negative or non-finite p makes later runs report GS_ENUMERIC.
 * Returns GS_EINVAL for a NULL context, GS_ECUDA if the launch fails.
 */
int gs_set_slm_amplitude(gs_ctx* c, const float* amplitude);

/*
 * gs_check_workspace -- verify the canary words of the context's workspace
 * (a diagnostic; the paper has no counterpart).
 *
 * Every buffer of the workspace is followed by 256 bytes of a fixed pattern,
 * written at creation; a kernel that wrote past the end of a buffer would
 * overwrite one. Synchronises the context stream and compares every canary.
 * Returns GS_OK, GS_ECORRUPT if one changed, GS_EINVAL for a NULL context,
 * GS_ECUDA on a CUDA error.
 */
int gs_check_workspace(gs_ctx* c);

/*
 * gs_test_corrupt_workspace -- test hook: overwrite one byte of the first
 * canary word from the host (a memset on the workspace; no kernel runs), so
 * that a test can see gs_check_workspace report GS_ECORRUPT. Returns GS_OK,
 * GS_EINVAL for a NULL context, GS_ECUDA on a CUDA error.
 */
int gs_test_corrupt_workspace(gs_ctx* c);

/*
 * gs_set_trace -- record per-pass timestamps of later runs (a diagnostic; the
 * paper reports per-iteration timings of its own FFT and constraint steps,
 * Sec. V, this is their counterpart for the fused passes).
 *
 * With enable != 0 every launch of gs_run / gs_run_batched on this context
 * writes, for each block, the globaltimer (ns) at the launch start and, for
 * each pass, when the block finished its work and when the grid barrier
 * released it. The record lives in the workspace; gs_get_trace reads the
 * last launch's. Costs two stores per pass and block. Returns GS_EINVAL for
 * a NULL or mixed context or enable < 0.
 */
int gs_set_trace(gs_ctx* c, int enable);

/*
 * gs_get_trace -- the timestamps of the last traced launch.
 *
 * Synchronises the context stream and copies (passes + 1) x grid pairs of
 * unsigned 64-bit nanosecond stamps to host_out, row-major: row 0 holds each
 * block's launch start (twice), row 1 + q pass q's (work done, released) per
 * block. *passes and *grid receive the shape (0 if nothing was traced).
 * Returns GS_EINVAL for NULL pointers, a mixed context or a capacity (in
 * stamps) below 2 (passes + 1) grid; GS_ECUDA on a CUDA error.
 */
int gs_get_trace(gs_ctx* c, unsigned long long* host_out, int capacity, int* passes, int* grid);

/*
 * gs_set_mask_group -- how many masks of a batched or mixed run are iterated
 * together (a tuning knob; the paper has no counterpart).
 *
 * A batch runs group after group, each group through the whole iteration
 * schedule of the launch, so that a group's fields (12 bytes per pixel) can
 * stay in L2; results do not depend on it (phases bit-identical, gaps to
 * FP64 rounding). masks = 0 (the default) takes, per grid size, the most
 * masks whose fields fit 100 MiB (8 of 1024 x 1024); masks > 0 fixes the
 * group size, capped by the batch. In a mixed run the sizes always run one
 * after the other. Returns GS_EINVAL for a NULL context or masks < 0.
 */
int gs_set_mask_group(gs_ctx* c, int masks);

/*
 * gs_set_grid -- tuning knob: number of thread blocks of the iteration kernel.
 *
 * ctas = 0 restores the automatic choice. A value above what the device can
 * keep resident at once is clamped. Host-only; takes effect at the next run.
 * A fixed grid also runs small grids on the persistent kernel (see gs_run).
 * Returns GS_EINVAL for a NULL context or ctas < 0.
 */
int gs_set_grid(gs_ctx* c, int ctas);

/*
 * gs_test_barrier_timeout -- test hook for the bounded device-side waits.
 *
 * The paper has no counterpart (failure detection of this library). With
 * enable != 0, every grid barrier of the context's later runs waits for one
 * arrival more than the grid provides, so the first barrier gives up after
 * its bounded wait (about 1 s), the run ends early with its outputs
 * unspecified, and gs_status reports GS_ETIMEOUT; the context stays usable.
 * enable = 0 restores normal runs. Host-only. Returns GS_EINVAL for a NULL
 * context or a negative enable.
 */
int gs_test_barrier_timeout(gs_ctx* c, int enable);

/*
 * gs_get_grid -- the number of thread blocks the next run will launch.
 * Writes it to *ctas (host). Returns GS_EINVAL for NULL arguments.
 */
int gs_get_grid(gs_ctx* c, int* ctas);

/*
 * gs_destroy -- free the context and its workspace. Synchronises the
 * context stream first. NULL is accepted (no-op). Returns GS_OK or GS_ECUDA.
 */
int gs_destroy(gs_ctx* c);

/*
 * gs_loss_grad -- intensity loss of a phase mask and its gradient.
 *
 * Operation: the differentiable form of the inverse problem of Sec. II (fit
 * the Fourier intensity of a phase-only field to the target):
 *   L(phi) = sum_k (|y_k|^2 / N - I_k)^2,   y = F exp(i phi)  (F unnormalised)
 *   dL/dphi = 4 Im(conj(x) * F^{-1}(r * y)),  x = exp(i phi), r = |y|^2/N - I,
 * F^{-1} the normalised inverse (the adjoint is computed by hand-written
 * passes, not by differentiating the forward code). Square grids only
 * (nx == ny), batch 1, on the context's workspace and stream. With an SLM
 * amplitude set (gs_set_slm_amplitude) the field is x = p exp(i phi).
 *   target_intensity  device, float [n][n], finite (any sign).
 *   phase             device, float [n][n], radians.
 *   loss_out          device, double[1].
 *   grad_out          device, float [n][n] (dL/dphi), or NULL for the loss only.
 * Asynchronous. Returns GS_EINVAL for NULL arguments or a non-square context,
 * GS_ECUDA if the launch fails; a non-finite target sets loss_out to NaN and
 * gs_status reports GS_ENUMERIC.
 */
int gs_loss_grad(gs_ctx* c, const float* target_intensity, const float* phase, double* loss_out, float* grad_out);

/*
 * gs_loss_prepare -- stage a target for repeated gs_loss_grad_prepared calls
 * (an optimisation over many steps with the same target).
 *
 * Operation: the target half of gs_loss_grad, once: checks that every value
 * is finite, reduces sum I and max I in FP64 and stores the target
 * transposed in the context's workspace, where the loss passes read it
 * column block by column block.
 *   target_intensity  device, float [n][n]; may be freed once the context's
 *                     stream has passed this call (the context keeps a copy).
 * Square grids only. Asynchronous. A non-finite target makes gs_status report
 * GS_ENUMERIC and later gs_loss_grad_prepared calls write NaN losses. The
 * staged target is overwritten (and later prepared calls refused) by any
 * gs_run / gs_run_batched, gs_loss_grad or gs_physical_error on the same
 * context. Returns GS_EINVAL for NULL arguments or a non-square context,
 * GS_ECUDA if the launch fails.
 */
int gs_loss_prepare(gs_ctx* c, const float* target_intensity);

/*
 * gs_loss_grad_prepared -- gs_loss_grad on the target of the last
 * gs_loss_prepare of this context: the same loss L(phi) and gradient, from
 * the three transform passes only (no validation or transposition of the
 * target per call). Arguments and layouts as gs_loss_grad. Returns GS_EINVAL
 * for NULL arguments, a non-square context or a context without a staged
 * target; GS_ECUDA if the launch fails.
 */
int gs_loss_grad_prepared(gs_ctx* c, const float* phase, double* loss_out, float* grad_out);

/*
 * gs_loss_adam_prepared -- one step of the phase optimiser in one launch:
 * gs_loss_grad_prepared followed by gs_adam_step, with the update applied in
 * the pass that forms the gradient (which is not stored).
 *   phase      device, float [n][n]: the phase phi of L(phi), updated in place.
 *   m, v       device, float [n][n]: the running moments of gs_adam_step.
 *   state      device, int [2] as in gs_adam_step (zero before the first step).
 *   lr, beta1, beta2, eps   as in gs_adam_step.
 *   loss_out   device, double [1]: L(phi) before the update.
 * The update is that of gs_adam_step with the gradient of
 * gs_loss_grad_prepared. Asynchronous. Returns GS_EINVAL as
 * gs_loss_grad_prepared and gs_adam_step do; GS_ECUDA if the launch fails.
 */
int gs_loss_adam_prepared(gs_ctx* c, float* phase, float* m, float* v, int* state, float lr, float beta1,
                          float beta2, float eps, double* loss_out);

/*
 * gs_loss_adam_run -- `steps` steps of the phase optimiser, each the step of
 * gs_loss_adam_prepared, with up to 1024 steps per launch.
 *
 * The same arithmetic as `steps` calls of gs_loss_adam_prepared in a row
 * (bit-identical losses, phase and moments), organised differently: within a
 * launch the pass that applies a step's update also forms the next step's
 * row transforms of exp(i phase), so a step costs two grid passes and two
 * grid barriers instead of a launch of three passes.
 *   phase, m, v, state, lr, beta1, beta2, eps   as gs_loss_adam_prepared.
 *   steps      >= 1.
 *   loss_out   device, double [steps]: loss_out[k] = L(phi) before step k.
 * The phase, m, v and state must not be written by anyone else until the
 * call's work on the context's stream is done. Asynchronous. Returns
 * GS_EINVAL as gs_loss_adam_prepared does or for steps < 1; GS_ECUDA if a
 * launch fails. A non-finite staged target writes NaN losses and leaves
 * phase, moments and state unchanged (gs_status reports GS_ENUMERIC).
 */
int gs_loss_adam_run(gs_ctx* c, float* phase, float* m, float* v, int* state, float lr, float beta1, float beta2,
                     float eps, int steps, double* loss_out);

/*
 * gs_physical_error -- the physical error of a phase mask, Eq. (phys-error).
 *
 * Operation: for the field u = p exp(i phase) on the SLM (p from
 * gs_set_slm_amplitude, else 1) and the target intensity I, with
 * It = I / max I and the reconstructed intensity
 * Ir = |F_u u|^2 (sum I / sum p^2) / max I (F_u the unitary DFT):
 *   E_l = sum over I > 0 of (t_d |It - Ir| / (t_l It) - t_d) Theta(|It - Ir|/It - t_l)
 *   E_d = sum over I = 0 of (Ir - t_d) Theta(Ir - t_d),   t_l = 0.1, t_d = 3e-4
 * (Sec. II: violations of the relative tolerance on lit pixels and the
 * absolute tolerance on dark pixels, summed in multiples of t_l and t_d; the
 * normalisation of Ir is this library's reading of a garbled passage).
 * Square grids only, on the context's workspace and stream.
 *   target_intensity  device, float [n][n], finite, >= 0, not all zero.
 *   phase             device, float [n][n], radians (e.g. a gs_run result).
 *   error_out         device, double[2] = (E_l, E_d).
 * Asynchronous. Returns GS_EINVAL for NULL arguments or a non-square context,
 * GS_ECUDA if the launch fails; a non-finite target gives NaN and GS_ENUMERIC.
 */
int gs_physical_error(gs_ctx* c, const float* target_intensity, const float* phase, double* error_out);

/*
 * gs_adam_step -- one Adam update of a phase mask from the gradient of the
 * intensity loss (gs_loss_grad): the optimiser of the differentiable form.
 * The paper iterates projections and has no optimiser; this is Adam (Kingma
 * and Ba, 2015) with bias correction, the form torch's Adam computes:
 *   m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
 *   phase -= (lr / (1 - beta1^t)) m / (sqrt(v / (1 - beta2^t)) + eps).
 *   phase, m, v  device float[n], updated in place (m, v zero before step 1).
 *   grad         device float[n].
 *   state        device int[2], zero before step 1: state[0] is the number
 *                of steps done (t - 1 during the call, t after it), state[1]
 *                an internal counter; both live on the device, so that the
 *                call can be captured once in a CUDA graph and replayed.
 *   lr > 0, 0 <= beta1, beta2 < 1, eps > 0.
 *   stream       a cudaStream_t or NULL. Asynchronous.
 * Returns GS_EINVAL for NULL arrays, n < 1 or bad hyperparameters; GS_ECUDA
 * if the launch fails.
 */
int gs_adam_step(float* phase, const float* grad, float* m, float* v, long long n, int* state, float lr,
                 float beta1, float beta2, float eps, void* stream);

/*
 * gs_run_noalloc -- gs_run without a context and without any allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory. A closed-loop stimulation controller cannot
 * afford cudaMalloc between spikes (it can synchronise the device and take
 * milliseconds); a host application may own all device memory through its
 * own pools and forbid libraries from calling the CUDA allocator; code
 * certified to allocate nothing after start-up cannot create a context.
 * This call performs the same operation as gs_run (same argument meaning,
 * layout and results) with the library's own static scratch instead of a
 * context workspace, and calls no cudaMalloc, cudaFree or allocating routine.
 * It always runs the persistent kernel with gs_run's automatic grid (one
 * block per 4096 pixels, small grids up to 32 blocks), also for the grids of
 * at most 8192 pixels that gs_run hands to its one-block-per-mask kernel:
 * the iterates are the same, such a small grid only runs slower here.
 *   nx, ny          powers of two in [32, 4096] with nx * ny <= 262144
 *                   (512 x 512): the static scratch holds one such grid.
 *                   Larger grids return GS_EINVAL (use gs_create/gs_run).
 *   flags, stream   as for gs_create (stream NULL = legacy default stream).
 *   target_intensity, phase_in, iters, phase_out, residual_out,
 *   object_gap_out  as for gs_run (device pointers owned by the caller).
 *   device_status   device int, or NULL: receives the device-side status of
 *                   this call (GS_OK, GS_ENUMERIC, GS_ETIMEOUT) once the
 *                   stream reaches it.
 * Scratch: about 4 MiB of device memory in a static array that every GPU which
 * loads the library holds until the process exits. All calls on a device
 * share it and it keeps the previous call's contents (each call clears what
 * must start at zero); calls whose work overlaps on the GPU (different
 * streams, or different host threads without ordering) race and corrupt each
 * other's results: serialise them on one stream. The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.
 * Asynchronous on `stream`. Returns GS_EINVAL for unsupported sizes or flags,
 * NULL arrays or iters < 0, GS_ECUDA if a CUDA call or launch fails.
 */
int gs_run_noalloc(int nx, int ny, unsigned flags, void* stream, const float* target_intensity,
                   const float* phase_in, int iters, float* phase_out, double* residual_out,
                   double* object_gap_out, int* device_status);

/*
 * gs_fp32_peak -- measured FP32 fused multiply-add throughput of the current
 * device (a diagnostic; the paper has no counterpart).
 *
 * Launches a kernel of independent FMA chains on every SM (as many blocks
 * as stay resident), times it with CUDA events on `stream` (a cudaStream_t,
 * or NULL for the legacy default stream) and writes 2 x FMAs / second in
 * TFLOP/s to *tflops_out (host), the best of three timed launches after one
 * warm-up. The denominator of the FP32 roofline of the iteration kernels.
 * Synchronous (waits for the timed launches). Returns GS_EINVAL for a NULL
 * tflops_out, GS_ECUDA if a CUDA call fails.
 */
int gs_fp32_peak(double* tflops_out, void* stream);

/*
 * gs_stream_notify -- wake a host thread when a stream reaches this point
 * (serving utility; the paper has no counterpart).
 *
 * Enqueues on `stream` (a cudaStream_t, or NULL for the legacy default
 * stream) a host function that writes the 8-byte value 1 to the file
 * descriptor `fd` (an eventfd or a pipe owned by the caller) once all work
 * enqueued before it on that stream has finished. A request loop can then
 * sleep in select/poll on `fd` until a launch completes or the next request
 * arrives, instead of spinning on events. The write happens on a thread of the
 * CUDA driver; the descriptor must stay open until it has run. Asynchronous.
 * Returns GS_EINVAL for fd < 0, GS_ECUDA if the host function cannot be
 * enqueued.
 */
int gs_stream_notify(void* stream, int fd);

/*
 * Persistent server (serving; the paper has no counterpart): one cooperative
 * launch that keeps iterating Eq. (e:AP) for the requests posted to its slots
 * and admits a request between two iterations of the others (continuous
 * batching with no host step between iterations). A request is the call of
 * gs_run for one n x n mask (n = 256, 512 or 1024; requests of different
 * sizes run together), p = 1, random-phase start: K iterations from
 * phase_in, phase_out and r^nu, g^nu (nu < K; no final residual) out. A
 * request of K iterations takes K + 1 server iterations (the first computes
 * the amplitude of Eq. pattern-constraint and u^0).
 *
 * Every buffer of a request is pinned host memory (cudaHostAlloc, or a
 * registered range) that the device reads and writes in place: the target
 * intensity and start phase ([n][n] row-major FP32) are read by the server,
 * the final phase ([n][n], may alias phase_in) and r, g (K doubles each, or
 * NULL) written by it. The caller keeps them alive and leaves them alone until
 * gs_serve_poll reports the request done. A server, like a context, is not
 * thread-safe: one host thread posts and polls.
 */
typedef struct gs_server gs_server;

/*
 * gs_serve_create -- a server for grids up to max_n x max_n (max_n = 256, 512
 * or 1024) with `slots` request slots (1..16) on `stream` (a cudaStream_t;
 * NULL: the legacy default stream, which the server then occupies while it
 * runs). `grid` is the number of blocks of its launches (0: one per SM; each
 * SM holds at most one), so two servers on two streams can share the device
 * by SM counts whose sum does not exceed it. Allocates the slot arrays
 * (12 max_n^2 bytes per slot) and the request table; launches nothing.
 * Returns GS_EINVAL for bad arguments, GS_ENOMEM, GS_ECUDA.
 */
int gs_serve_create(gs_server** out, int max_n, int slots, int grid, void* stream);

/*
 * gs_serve_submit -- post a request of `iters` >= 1 iterations for an n x n
 * grid (n = 256, 512 or 1024, at most max_n) to slot `slot`, which must be
 * free (its previous request reported done). Writes the
 * request and its sequence number (returned in *seq_out, nonzero, if not
 * NULL) to the table and launches the server if no launch is serving. Returns
 * GS_EINVAL for a busy slot, a bad argument or a buffer the device cannot
 * address, GS_ECUDA if the launch fails, or the server's failure status.
 */
int gs_serve_submit(gs_server* s, int slot, int n, const float* target_intensity, const float* phase_in,
                    int iters, float* phase_out, double* residual_out, double* object_gap_out, unsigned* seq_out);

/*
 * gs_serve_poll -- the sequence number of the last request of `slot` that is
 * done (*done_seq; the request's outputs are complete once it equals the
 * submitted one) and that request's status (*request_status: GS_OK,
 * GS_ENUMERIC for a target with a negative, non-finite or all-zero
 * intensity, GS_EINVAL). Relaunches the server when requests are outstanding
 * and no launch runs (a launch leaves after 20 ms without work, and after
 * 2^20 iterations). Non-blocking. Returns GS_OK, or the server's failure
 * status (e.g. GS_ETIMEOUT from a grid barrier), after which no request
 * completes.
 */
int gs_serve_poll(gs_server* s, int slot, unsigned* done_seq, int* request_status);

/*
 * gs_serve_stop -- block until every posted request is done and no launch
 * runs. Returns GS_OK, the server's failure status, or GS_ETIMEOUT if
 * requests were still outstanding after 60 s.
 */
int gs_serve_stop(gs_server* s);

/* gs_serve_grid -- blocks per launch of the server (0 for NULL). */
int gs_serve_grid(const gs_server* s);

/*
 * gs_serve_test_tick_limit -- test hook: a launch leaves after `ticks`
 * iterations (1..2^20; 2^20 by default) even with requests running, which the
 * next launch resumes. Only while no launch runs; GS_EINVAL otherwise.
 */
int gs_serve_test_tick_limit(gs_server* s, int ticks);

/* gs_serve_destroy -- stop, then free the server. NULL is a no-op. */
void gs_serve_destroy(gs_server* s);

/* gs_strerror -- static English text for a status code (never NULL). */
const char* gs_strerror(int code);

/*
 * gs_workspace_bytes -- device bytes a context for nx x ny allocates
 * (for admission by memory). Pure host computation; 0 for invalid sizes.
 */
size_t gs_workspace_bytes(int nx, int ny, unsigned flags);

/*
 * gs_workspace_bytes_batched -- device bytes of a gs_create_batched context
 * (for admission by memory). Pure host computation; 0 for invalid arguments.
 */
size_t gs_workspace_bytes_batched(int nx, int ny, int max_batch, unsigned flags);

#ifdef __cplusplus
}
#endif

#endif /* GS_GB300_H */
