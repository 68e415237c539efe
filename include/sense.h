/*
 * libsense — C ABI of the B300 SENSE / unrolled-reconstruction hot path.
 *
 * Operations follow Blumenthal et al., "Deep, Deep Learning with BART":
 *   Eq. 4 ("inverse_problem", Sec. 2.3): A = P F C — coil-sensitivity multiply
 *     (C), centred unitary 2-D Fourier transform (F), sampling projection (P).
 *   Eq. 6 ("update_modl", Sec. 2.3.2): the MoDL data-consistency step applies
 *     S_lambda^{-1} = (A^H A + lambda I)^{-1} with conjugate gradients; the
 *     derivatives of S^{-1} are written through S itself (same section).
 *   Eq. 5 ("update_vn", Sec. 2.3.1): the VarNet step uses A^H A x - A^H y.
 *
 * Conventions shared by every call
 *   - Complex data are complex64: interleaved (re, im) float32, 8 bytes.
 *   - Layouts are row-major, W fastest:
 *       image x     [B][H][W]
 *       maps S      [B][C][H][W]     (one set of maps per slice)
 *       k-space y   [B][C][H][W]     full Cartesian grid, centred (DC at H/2, W/2)
 *       mask M      [W] (line mask: constant along H; mask_is_lines = 1)
 *                   or [H][W] (mask_is_lines = 0), float32, centred order.
 *     The normal operator uses M^2 (P^H P); for 0/1 masks that is M.
 *   - Every data pointer is a DEVICE pointer owned by the caller and must be
 *     16-byte aligned; the library never frees caller memory.  A plan keeps
 *     the maps and mask pointers it was created with (no copy): the caller
 *     keeps them alive and unchanged for the plan's lifetime.
 *   - Calls are asynchronous on the plan's CUDA stream; results are ready
 *     when that stream reaches them.  A plan is not thread-safe.  Some calls
 *     (the MoDL denoiser backward, the VarNet stages) also run independent
 *     parts on three side streams the library creates per device on first
 *     use, forked from and joined back to the caller's stream with events, so
 *     their results are still ready in the caller's stream order (except where
 *     SENSE_VN_DEFER_JOIN says otherwise).  The side streams are shared by every
 *     plan and call on the device: calls made at the same time from different
 *     caller streams queue behind each other's side-stream work, and a stream
 *     capture of such a call must not overlap library calls from other threads
 *     on that device (their side-stream work would join the capture).
 *   - Return value: SENSE_OK (0) or a negative SENSE_E* code; host-side
 *     argument checks run before any launch, so an error leaves outputs
 *     untouched.  Device-side failures (CG breakdown, non-finite scalars) set
 *     bits of the plan's device status word, read by sense_get_status; the
 *     kernels never trap.
 *   - Even H and W are required (the centred transform uses the (-1)^n
 *     modulation of an even-length DFT).
 */
#ifndef SENSE_H
#define SENSE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SENSE_OK 0
#define SENSE_EINVAL_SHAPE (-1)   /* non-positive or odd size */
#define SENSE_EINVAL_PTR (-2)     /* NULL, aliased or misaligned pointer */
#define SENSE_EINVAL_LAMBDA (-3)  /* lambda not finite or negative */
#define SENSE_EUNSUPPORTED (-4)   /* shape the kernels do not cover (e.g. prime factor > 31) */
#define SENSE_ECUDA (-5)          /* a CUDA runtime call failed */
#define SENSE_EWORKSPACE (-6)     /* workspace missing or too small */
#define SENSE_EINVAL_ARG (-7)     /* other invalid argument (iteration count, flags) */
#define SENSE_ETOO_LARGE (-8)     /* problem larger than the fixed scratch of sense_dot_re_noalloc */

/* Device status bits (sense_get_status). */
#define SENSE_STATUS_CG_BREAKDOWN 1 /* Re<p, S p> <= 0 on a slice with nonzero residual */
#define SENSE_STATUS_NONFINITE 2    /* a CG scalar became NaN or Inf */
#define SENSE_STATUS_DEVICE_TIMEOUT 4 /* a bounded wait inside a kernel gave up (work skipped) */

typedef struct sense_plan_s* sense_plan;

/* Create a plan for B slices of C coils on an H x W grid.
 * maps: device complex64 [B][C][H][W]; mask: device float32 [W] or [H][W];
 * stream: cudaStream_t (NULL = legacy default stream).
 * The mask is copied to the host once here (synchronously) to build the
 * pruned-transform tables; later changes to it are not seen.
 * Errors: SENSE_EINVAL_SHAPE, SENSE_EINVAL_PTR, SENSE_EUNSUPPORTED, SENSE_ECUDA. */
int sense_plan_create(sense_plan* plan, int B, int C, int H, int W, const void* maps,
                      const float* mask, int mask_is_lines, void* stream);
/* Soft-SENSE (Sec. 2.3.3, "Extensions to the SENSE model"): S >= 1 sets of maps,
 * maps [B][S][C][H][W].  Every image of such a plan (x, x0, rhs, out, AHy, CG
 * vectors) is [B][S][H][W], one component per map set:
 *   A x = { M F sum_s S_{s,c} x_s }_c,   (A^H y)_s = sum_c conj(S_{s,c}) F^{-1}(M y_c).
 * S = 1 is sense_plan_create.  S = 2 with a line mask uses the fused
 * normal-operator kernel where one is compiled (W = 128, 232, 320, 368); other
 * cases (S <= 8) run the generic row/column transforms.  The learned-regulariser
 * calls (unrolled_step, varnet_stage, ...) take S = 1 plans only
 * (SENSE_EUNSUPPORTED). */
int sense_plan_create_sets(sense_plan* plan, int B, int S, int C, int H, int W, const void* maps,
                           const float* mask, int mask_is_lines, void* stream);
/* Non-Cartesian SENSE (Sec. 2.3.3): the normal operator A^H A is applied as a
 * convolution with the point spread function of the sampling pattern (the
 * Toeplitz embedding on the 2H x 2W grid); A^H y is precomputed by the caller,
 * as in the paper.  psf: device complex64 [2H][2W] as sense_toeplitz_psf
 * writes it; the plan transforms it once at creation (asynchronously on
 * stream) and keeps its own copy.  Such a plan supports sense_normal,
 * cg_dc_solve(_backward), the unrolled blocks and varnet_stage (images
 * [B][H][W]); sense_forward and sense_adjoint return SENSE_EUNSUPPORTED.
 * The workspace holds [B][C][H][2W] coil rows. */
int sense_plan_create_toeplitz(sense_plan* plan, int B, int C, int H, int W, const void* maps,
                               const void* psf, void* stream);
/* PSF of a non-Cartesian trajectory on the 2H x 2W embedding grid (direct sum
 * over the M samples: FP32 phasors, FP64 accumulation):
 *   psf[iy][ix] = (H W)^{-1} sum_m exp(2 pi i (ky_m dy / H + kx_m dx / W)),
 *   dy = iy (iy < H) or iy - 2H, dx likewise; zero on row H and column W.
 * traj: device float32 [M][2] = (ky, kx) in grid units (the Cartesian grid is
 * the integer lattice, k in [-H/2, H/2) x [-W/2, W/2)); image coordinates are
 * centred (index - H/2, index - W/2), so on-grid samples give the centred
 * unitary DFT of sense_forward.  psf: device complex64 [2H][2W]. */
int sense_toeplitz_psf(const float* traj, int M, int H, int W, void* psf, void* stream);
/* Non-uniform DFT pair of non-Cartesian SENSE by direct summation (Sec. 2.3.3: the adjoint of
 * the measured non-Cartesian samples initialises the networks, x^0 = A^H y):
 *   forward  y[b][c][m] = (H W)^{-1/2} sum_n S_c(n) x(n) exp(-2 pi i (ky_m n'_y / H + kx_m n'_x / W))
 *   adjoint  x[b][n]    = (H W)^{-1/2} sum_c conj(S_c(n)) sum_m y[b][c][m] exp(+2 pi i (...))
 * n' = n - (H/2, W/2) (centred image coordinates), traj as for sense_toeplitz_psf, so on-grid
 * samples give the centred unitary DFT of sense_forward and A^H A equals the Toeplitz-embedded
 * normal operator of the PSF.  maps complex64 [B][C][H][W], x [B][H][W], y [B][C][M] (device,
 * 8-byte aligned; x and y must not alias).  Cost O(M H W C) per slice (set-up calls, like the
 * PSF).  Asynchronous on stream.  Errors: SENSE_EINVAL_SHAPE, SENSE_EINVAL_PTR,
 * SENSE_EUNSUPPORTED (H or W > 4096). */
int sense_nudft_forward(const float* traj, int M, int B, int C, int H, int W, const void* maps,
                        const void* x, void* y, void* stream);
int sense_nudft_adjoint(const float* traj, int M, int B, int C, int H, int W, const void* maps,
                        const void* y, void* x, void* stream);
int sense_plan_destroy(sense_plan plan);
/* Change the stream later calls launch on. */
int sense_plan_set_stream(sense_plan plan, void* stream);

/* Scratch memory the plan needs for the calls below (bytes).  The caller
 * allocates it on the device (256-byte aligned) and hands it over once; the
 * plan uses it until destroyed or given another one.  Calls that overlap in
 * time on different streams must not share one plan. */
int sense_plan_workspace_bytes(sense_plan plan, size_t* bytes);
int sense_plan_set_workspace(sense_plan plan, void* workspace, size_t bytes);

/* y = P F C x (Eq. 4).  x [B][H][W] -> y [B][C][H][W] (zero where M = 0). */
int sense_forward(sense_plan plan, const void* x, void* y);

/* x = A^H y = sum_c conj(S_c) F^{-1}(M y_c)  (adjoint of Eq. 4; A^H y is the
 * initialisation x^0 of both MoDL and VarNet, Sec. 2.3.1-2.3.2).
 * Needs the workspace. */
int sense_adjoint(sense_plan plan, const void* y, void* x);

/* out = (A^H A + lambda I) x, the operator S_lambda of Eq. 6 (lambda >= 0,
 * finite).  x and out must not alias.  Fused per-row kernel for line masks
 * (no workspace); 2-D masks go through the workspace. */
int sense_normal(sense_plan plan, const void* x, void* out, float lambda);

/* x = S_lambda^{-1} rhs by exactly `iters` conjugate-gradient iterations
 * (Sec. 2.3.2), independently per slice.
 *   rhs    [B][H][W]
 *   x0     [B][H][W] start value, or NULL for zero
 *   x      [B][H][W] output (may alias x0, must not alias rhs)
 *   lambda device float64, lambda_count = 1 (shared) or B (per slice), > 0
 *          (not checked on the host: lambda <= 0 shows up as a breakdown bit)
 *   rr_hist NULL or device float64 [iters + 1][B]: ||r_i||^2 per iteration.
 * Vectors are FP32 complex; alpha and beta are FP64.  Inner products take FP32
 * products and lane sums, summed across lanes and rows in FP64 or (the one-launch
 * solve on line masks) as compensated float-float pairs converted to FP64 once.
 * A slice whose residual is exactly zero is frozen.  Needs the workspace. */
int cg_dc_solve(sense_plan plan, const void* rhs, const void* x0, void* x,
                const double* lambda, int lambda_count, int iters, double* rr_hist);

/* Reverse mode of the MoDL data-consistency block x = S^{-1}(b + lambda z)
 * (derivative identities of S^{-1}, Sec. 2.3.2):
 *   grad_rhs    = v = S^{-1} grad_x            (second CG solve, x0 = 0)
 *   grad_lambda = Re<v, z - x>  (summed over slices if lambda_count = 1, else per slice)
 * grad_x, x, z: [B][H][W]; z may be NULL (rhs independent of lambda: -Re<v, x>).
 * grad_lambda: NULL or device float64 [lambda_count], overwritten.
 * Complex gradients follow Sec. 2.2.2: real part = d/d(re), imaginary = d/d(im).
 * Needs the workspace. */
int cg_dc_solve_backward(sense_plan plan, const void* grad_x, const void* x, const void* z,
                         const double* lambda, int lambda_count, int iters,
                         void* grad_rhs, double* grad_lambda);

/* Profiling (process-wide).  The library counts every kernel it launches;
 * with enable != 0 it also records a CUDA event pair on the launching stream
 * around each launch of its main kernels, grouped by name: "normal_lines"
 * (fused normal operator), "conv64_tc" (tensor-core convolution), "wgrad64"
 * (64-channel weight gradient). */
int sense_profile_enable(int enable);
/* Summed event time (ms) and number of timed launches of one kernel group
 * since its last read (waits for the recorded events); resets the group. */
int sense_profile_read(const char* name, double* ms, int* launches);
/* Kernels launched so far (reset to zero if reset != 0). */
long long sense_kernel_launches(int reset);
/* Measurement aid (no counterpart in the paper): a register-only FP32 FMA kernel of `blocks`
 * blocks of 256 threads, each thread running 8 independent chains of `iters` FMAs
 * (2 * 8 * 256 * iters FLOP per block), for timing the FP32 pipe's peak with CUDA events on
 * `stream`.  sink: device float32 [blocks] (written only in a practically unreachable case). */
int sense_fma_probe(int blocks, int iters, float* sink, void* stream);

/* Synchronises the plan's stream, returns the OR of device status bits set
 * since the last call, and clears them. */
int sense_get_status(sense_plan plan, int* device_status);

/* Failure detection (no counterpart in the paper): the bounded waits of the
 * one-launch CG.  Each CTA of that kernel waits at one barrier per CG pass
 * for the other CTAs of its slice, polling a release word at most `polls`
 * times (0 restores the default, 2^22 polls of about 32 ns plus the load);
 * a CTA that gives up sets SENSE_STATUS_DEVICE_TIMEOUT, skips the rest of the
 * solve and returns, so the kernel always ends and the context stays usable.
 * unreachable = 1 makes every barrier expect one arrival that never comes, so
 * every wait runs out (this exists to test the timeout path; the solve's
 * result is then undefined); 0 is normal operation.  Host-side only; applies
 * to later calls of this plan.  Errors: SENSE_EINVAL_PTR, SENSE_EINVAL_ARG. */
int sense_plan_set_wait_limit(sense_plan plan, unsigned polls, int unreachable);

/* ------------------------------------------------------------------------
 * Learned denoisers.  SENSE_DENOISER_MODL: the MoDL residual CNN
 * D_W(x) = x + CNN(x) (Sec. 2.3.2, Eq. 6) with 3x3 convolutions
 * 2 -> 64 -> 64 -> 64 -> 64 -> 2 (biases, ReLU between layers, no batch norm);
 * the complex image enters as two real channels (re, im).
 * SENSE_DENOISER_VARNET: the VarNet regulariser term of Eq. 5 (Sec. 2.3.1),
 * R(x) = sum_i K_i^T Phi_i'(K_i x), with the filters and RBF weights of one
 * stage in the layout of varnet_stage below (6,553 values; lambda_t unused);
 * its workspace is varnet's (no status word; backward always recomputes K x).
 *
 * weights: device float32, denoiser_param_count() values, layer by layer
 *   w_l [Cout][Cin][3][3] then b_l [Cout], l = 1..5 (113,154 for MoDL).
 * Convolutions are cross-correlations with zero "same" padding.  Activations
 * are stored in BF16 (channels-last), products accumulate in FP32; the
 * network input is rounded to BF16.  The 64 -> 64 layers run on the tensor
 * cores (tcgen05, FP32 accumulators in tensor memory).
 *
 * ws: device workspace of denoiser_workspace_bytes() bytes, 256-byte
 *   aligned, zero-filled by the caller once before first use (it holds the
 *   status word read by denoiser_get_status).  It keeps the activations of
 *   the last forward call, so denoiser_backward(recompute = 0) may follow a
 *   denoiser_forward on the same x and ws without recomputing them
 *   (recompute = 1 reruns the forward first: the recomputation policy of the
 *   checkpointing container, Sec. 2.2.4).  Calls sharing a ws must not overlap.
 */
#define SENSE_DENOISER_MODL 0
#define SENSE_DENOISER_VARNET 1
size_t denoiser_workspace_bytes(int kind, int B, int H, int W);
int denoiser_param_count(int kind);
/* MoDL: byte offsets inside ws of the four BF16 [B][H][W][64] layer activations
 * and the two BF16 gradient buffers (for inspection and per-layer checks). */
int denoiser_workspace_offsets(int kind, int B, int H, int W, size_t* act_offsets,
                               size_t* grad_offsets);
/* out = D_W(x) (MoDL) or R(x) (VarNet); x, out complex64 [B][H][W] (must not alias). */
int denoiser_forward(int kind, const float* weights, const void* x, void* out, void* ws,
                     size_t ws_bytes, int B, int H, int W, void* stream);
/* Reverse mode: grad_x = (dD/dx)^H grad_out (complex convention of Sec. 2.2.2)
 * and grad_weights += dL/dW (float32, same layout as weights; accumulated so
 * that blocks sharing weights add up; deterministic fixed-order sums). */
int denoiser_backward(int kind, const float* weights, const void* x, const void* grad_out,
                      void* grad_x, float* grad_weights, void* ws, size_t ws_bytes, int B, int H,
                      int W, int recompute, void* stream);
/* MoDL workspaces: reads (synchronising the stream) and clears the status word in ws. */
int denoiser_get_status(void* ws, int B, int H, int W, void* stream, int* device_status);

/* ------------------------------------------------------------------------
 * Unrolled block on a plan (maps, mask, workspace) and a denoiser workspace,
 * on the plan's stream.  x_t, x_next, AHy, grad_next, grad_t: complex64 [B][H][W].
 * kind SENSE_DENOISER_MODL (Eq. 6, Sec. 2.3.2); lambda: device float64 [1]:
 *   unrolled_step:  z = D_W(x_t);  x_next = S_lambda^{-1}(AHy + lambda z) by
 *                   cg_iters CG iterations from zero; z and the denoiser activations
 *                   stay in dn_ws.
 *   unrolled_step_backward: given grad_next = dL/dx_next, recomputes z from x_t
 *                   (checkpointing, Sec. 2.2.4), solves v = S_lambda^{-1} grad_next,
 *                   adds Re<v, z - x_next> to grad_lambda[0], and writes
 *                   grad_t = (dD/dx)^H (lambda v) while adding dL/dW to grad_weights.
 * kind SENSE_DENOISER_VARNET (Eq. 5, Sec. 2.3.1): the calls are varnet_stage and
 *   varnet_stage_backward (lambda_t and its gradient live in the stage
 *   parameters; lambda, grad_lambda, x_next of the backward and cg_iters are
 *   not used; dn_ws is a varnet workspace). */
int unrolled_step(sense_plan plan, int kind, const float* weights, const double* lambda,
                  const void* AHy, const void* x_t, void* x_next, int cg_iters, void* dn_ws,
                  size_t dn_ws_bytes);
int unrolled_step_backward(sense_plan plan, int kind, const float* weights, const double* lambda,
                           const void* AHy, const void* x_t, const void* x_next,
                           const void* grad_next, void* grad_t, float* grad_weights,
                           double* grad_lambda, int cg_iters, void* dn_ws, size_t dn_ws_bytes);
/* The same with a choice (MoDL): recompute != 0 is unrolled_step_backward; recompute == 0 takes z
 * and the denoiser activations from dn_ws as the unrolled_step of this block left them (the
 * caller keeps one denoiser workspace per block between the forward and reverse passes, and
 * the weights unchanged) instead of recomputing them.  Results are identical either way. */
int unrolled_step_backward_ex(sense_plan plan, int kind, const float* weights, const double* lambda,
                              const void* AHy, const void* x_t, const void* x_next,
                              const void* grad_next, void* grad_t, float* grad_weights,
                              double* grad_lambda, int cg_iters, void* dn_ws, size_t dn_ws_bytes,
                              int recompute);

/* ------------------------------------------------------------------------
 * VarNet gradient stage (Eq. 5, Sec. 2.3.1) on a plan (maps, mask, workspace):
 *   x_next = x_t - sum_i K_i^T Phi_i'(K_i x_t) - lambda_t (A^H A x_t - A^H y)
 * with VARNET_NK complex 11x11 filters k_i, K_i x = Re(k_i * x) (a
 * cross-correlation with zero "same" padding; the imaginary part is
 * discarded) and Phi_i'(z) = sum_j r_ij exp(-(z - mu_j)^2 / (2 sigma^2)),
 * VARNET_NW centres mu_j = -1 + 2 j / (VARNET_NW - 1), sigma = their spacing.
 *
 * params: device float32 [varnet_param_count()] = 6,553 values per stage:
 *   w[i][c][dy][dx]  i < 24, c < 2, 11x11: w[i][0] = Re k_i, w[i][1] = -Im k_i
 *   r[i][j]          RBF weights, j < 31
 *   lambda_t         (last value)
 * AHy, x_t, x_next, grad_next, grad_t, nx: device complex64 [B][H][W], W <= 512.
 * Arithmetic: filters rounded to bfloat16 at use, float32 accumulation on the
 * tensor cores; K's image operand is split into two bfloat16 terms (hi + lo),
 * which makes K x as accurate as float32 accumulation (the zero-mean filters
 * cancel on smooth images, where one bfloat16 rounding of x would cost ~1e-2
 * relative); Phi'(K x) and Phi''(K x) K g are stored in bfloat16 for K^T and
 * the filter gradient.  Phi' sums the 13 centres nearest z (the rest are
 * below exp(-21) of the largest term).  A^H A as sense_normal.
 *
 *   varnet_stage:          writes x_next (x_next != x_t).  nx_out (optional,
 *       else NULL) receives A^H A x_t for the reverse pass.
 *   varnet_stage_backward: given grad_next = dL/dx_next writes
 *       grad_t = grad_next - K^T(Phi''(K x_t) K grad_next) - lambda_t A^H A grad_next
 *     and ADDS dL/dparams to grad_params (filters, RBF weights, lambda_t);
 *     grad_t != grad_next (grad_t may alias x_t).  nx_t: A^H A x_t as written
 *     by varnet_stage, or NULL to recompute it.  Needs the plan workspace.
 * ws: device workspace of varnet_workspace_bytes(B, H, W) bytes, 256-byte
 * aligned, used by one call at a time.  Gradient sums use a fixed order:
 * results are bitwise reproducible.  Plan's stream, asynchronous. */
#define VARNET_NK 24
#define VARNET_NW 31
#define VARNET_KSIZE 11
size_t varnet_workspace_bytes(int B, int H, int W);
int varnet_param_count(void);
/* Byte offsets in ws of the activations the last call left there (for tests and
 * inspection): offsets[0] u = Phi'(K x_t) and offsets[1] v = Phi''(K x_t) K grad_next,
 * bfloat16 [B][H][W][32] (channels 24..31 zero); offsets[2] z = K x_t and
 * offsets[3] K grad_next, float32 [B][H][W][24] (u and z from varnet_stage and a
 * recomputing varnet_stage_backward; v and K grad_next from varnet_stage_backward). */
int varnet_workspace_offsets(int B, int H, int W, size_t* offsets);
int varnet_stage(sense_plan plan, const float* params, const void* AHy, const void* x_t, void* x_next,
                 void* nx_out, void* ws, size_t ws_bytes);
int varnet_stage_backward(sense_plan plan, const float* params, const void* AHy, const void* x_t,
                          const void* nx_t, const void* grad_next, void* grad_t, float* grad_params,
                          void* ws, size_t ws_bytes);
/* The same with choices in `recompute` (bit flags):
 *   bit 0 (value 1): set = varnet_stage_backward (K x recomputed); clear = take z = K x and
 *     u = Phi'(z) from ws as varnet_stage of this stage left them (the caller keeps one varnet
 *     workspace per stage between the forward and reverse passes, parameters unchanged), so only
 *     K g is computed; results are the same.
 *   bit 1 (SENSE_VN_DEFER_JOIN): the parameter gradients of the stage (grad_params) may still be
 *     running on the library's side streams when the call's work on the plan's stream is done;
 *     grad_t is complete in stream order as always.  Until sense_streams_join(stream) has been
 *     called on the stream that reads them, the caller must not read grad_params nor change ws,
 *     x_t, grad_next or params.  A reverse pass over T stages with one workspace and one
 *     grad_next buffer per stage can so overlap each stage's parameter gradients with the next
 *     stage's work; the gradients are bitwise the same. */
#define SENSE_VN_DEFER_JOIN 2
int varnet_stage_backward_ex(sense_plan plan, const float* params, const void* AHy, const void* x_t,
                             const void* nx_t, const void* grad_next, void* grad_t, float* grad_params,
                             void* ws, size_t ws_bytes, int recompute);
/* Make `stream` (a cudaStream_t, NULL = the legacy default stream) wait for all work issued so far
 * on the library's side streams of the current device (see SENSE_VN_DEFER_JOIN).  Asynchronous;
 * SENSE_ECUDA if the wait cannot be enqueued.  No counterpart in the paper. */
int sense_streams_join(void* stream);

/* Training loss of the unrolled networks: loss[0] = mean |x - gt|^2 over the
 * plan's B*S*H*W complex elements (float64, fixed-order sum) and
 * grad = 2 (x - gt) / n (complex convention of Sec. 2.2.2).  Plan's stream. */
int sense_mse_loss(sense_plan plan, const void* x, const void* gt, double* loss, void* grad);

/* Per-slice data scaling of the VarNet workload (Sec. 2.3.1: the data are
 * scaled so that max |x^0| = 1): with m_b = max over slice b of |x_b|,
 * x_b /= m_b and, when other != NULL, other_b /= m_b (e.g. the ground truth of
 * the loss); scale (NULL or device float32 [B]) receives 1 / m_b.  An all-zero
 * slice is left as it is (scale 1).  x, other: complex64 [B][H][W].  Uses the
 * plan's workspace; plan's stream. */
int sense_normalize_max(sense_plan plan, void* x, void* other, float* scale);

/* Adam (Kingma and Ba) on n parameters with moments m, v; step >= 1 is the
 * 1-based update count (bias correction).  The gradient is consumed and set
 * to zero, ready to accumulate the next step.  The float64 variant clamps the
 * parameters at `lower` (used to keep the MoDL lambda positive). */
int adam_update_f32(float* param, float* grad, float* m, float* v, size_t n, float lr, float beta1,
                    float beta2, float eps, int step, void* stream);
int adam_update_f64(double* param, double* grad, double* m, double* v, size_t n, double lr,
                    double beta1, double beta2, double eps, int step, double lower, void* stream);

/* iPALM update of VarNet stage parameters (Sec. 2.3.1: the VarNet is trained with iPALM,
 * the inertial proximal alternating linearised minimisation of Pock and Sabach).  The paper
 * names neither the constraints nor the inertia; this call takes the variational-network
 * constraints (each complex filter zero-mean over its taps with Euclidean norm <= 1,
 * lambda_t >= 0, RBF weights free) and alpha = beta.  Update k of T stages in the layout of
 * varnet_stage (T * 6,553 float32 values each):
 *   on entry  params = z^k (the point where grad was taken), x = x^k;
 *   on exit   x = x^{k+1} = P(z^k - tau grad) blockwise (tau_filters, tau_rbf, tau_lambda),
 *             params = z^{k+1} = x^{k+1} + alpha_next (x^{k+1} - x^k),
 *             grad = 0 (ready to accumulate the next step).
 * Start with x = params (x^0 = z^1); the usual inertia is alpha_next = k / (k + 3).
 * params, grad and x must not alias.  Asynchronous on stream.  Errors: SENSE_EINVAL_PTR,
 * SENSE_EINVAL_ARG (T <= 0, negative or non-finite step sizes, alpha_next outside [0, 1)). */
int ipalm_update_varnet(float* params, float* grad, float* x, int T, float tau_filters,
                        float tau_rbf, float tau_lambda, float alpha_next, void* stream);

/* Allocation-free variant of the inner product behind the lambda gradient of
 * cg_dc_solve_backward.  The paper has no counterpart; it exists for callers
 * that must not allocate GPU memory once they are running — for example a
 * reconstruction service that reserves all device memory at start-up and
 * may not call cudaMalloc while data streams in (an allocation can stall the
 * device and every other stream on it), or a host program whose own memory
 * manager owns the device heap.  It needs no plan and no workspace:
 *
 *   out[b] = sum over slice b of Re<a, b_ - c>   (out_count = B), or the sum
 *            over all slices in slice order      (out_count = 1)
 *
 * a, b_, c: device complex64 [B][H][W], 16-byte aligned; b_ or c may be NULL
 * (read as zero).  W must be even.  out: device float64 [out_count].
 * stream: cudaStream_t (NULL = legacy default stream).  Asynchronous.
 *
 * Scratch: a fixed array of SENSE_NOALLOC_SCRATCH_BYTES in the library's own
 * device memory (every GPU that loads the library holds one copy until the
 * process exits).  It takes B * H <= SENSE_NOALLOC_MAX_ROWS; larger problems
 * get SENSE_ETOO_LARGE before anything runs.  The first call on each device
 * looks up the array's device address (with that device current), so make
 * that first call before any stream capture.  Later calls on a stream that is
 * not being captured look it up again, so an address that moved after
 * cudaDeviceReset is picked up.  Every call shares the array: calls that
 * overlap on the GPU (other streams, other host threads) race and give wrong
 * results — serialise them.  The rows are split and summed exactly as in the
 * workspace kernel of cg_dc_solve_backward (two warps per row, FP64 warp sums,
 * fixed-order slice sums), so the results equal that path's bit for bit. */
#define SENSE_NOALLOC_SCRATCH_BYTES (1u << 20)
#define SENSE_NOALLOC_MAX_ROWS ((SENSE_NOALLOC_SCRATCH_BYTES - 256u) / 8u)
int sense_dot_re_noalloc(int B, int H, int W, const void* a, const void* b_, const void* c,
                         double* out, int out_count, void* stream);

/* Static description of an error code (never NULL). */
const char* sense_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* SENSE_H */
