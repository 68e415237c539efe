// Internal plan state of libsense and the launcher declarations shared by the
// translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

#define SENSE_MAX_STAGES 24

// Tables of a 1-D transform of length L (generic mixed-radix path).
struct Fft1D {
  int L = 0;
  int nst = 0;
  int radix[SENSE_MAX_STAGES] = {0};
  float2* tw = nullptr;  // device [L], e^{-2 pi i m / L}
};

// Tables of the fused line-mask normal operator, W = Q * P (Q a power of two).
struct LinesTables {
  int ok = 0;
  int Q = 0, P = 0, J = 0, JMAX = 0;
  int kstride = 0;         // float4 quads per k1 block of the coefficient table
  int rows = 0, nwr = 0, threads = 0, smem = 0, grid = 0;
  float4* coef = nullptr;  // [Q][kstride]
  float2* tw = nullptr;    // [Q][P] e^{-2 pi i t k1 / W}
  float* wt = nullptr;     // [Q][J] mask^2 / W per slot (0 = padding)
  float* sgn = nullptr;    // [Q][J] (-1)^{k2} (even P only)
  int* akx = nullptr;      // [Q][J] adjoint: centred column index (k + W/2) mod W of slot (k1, j)
  float* af = nullptr;     // [Q][J] adjoint: (-1)^k / sqrt(W) per slot (0 = padding)
  int* cols = nullptr;     // sampled columns (centred index), ncols of them
  int ncols = 0;
  const void* coop = nullptr;  // whole-solve cooperative CG kernel (NULL: one launch per step)
  int coop_grid = 0;
};

// Scratch carved from the caller's workspace.
struct Workspace {
  float2* T = nullptr;          // [B][C][H][W] coil-image intermediate
  float2* r = nullptr;          // [B][H][W]
  float2* p = nullptr;
  float2* q = nullptr;
  float2* t0 = nullptr;         // [B][H][W] temporaries of the unrolled blocks
  float2* t1 = nullptr;
  double* part = nullptr;       // [B][H] per-row partial sums
  double* part2 = nullptr;      // [4][B][H] row partials of the one-launch CG (two double buffers)
  float2* wv = nullptr;         // [B][S][H][W] S r of the one-launch CG
  float2* sv = nullptr;         // [B][S][H][W] S p of the one-launch CG
  double* rr = nullptr;         // [B]  ||r||^2
  double* alpha = nullptr;      // [B]
  double* beta = nullptr;       // [B]
  double* lam = nullptr;        // [B]  lambda per slice (float64)
  unsigned* counter = nullptr;  // last-block counter (zero between kernels)
};

struct sense_plan_s {
  int B = 0, C = 0, H = 0, W = 0;
  int S = 1;                    // sets of maps (soft-SENSE); images are [B][S][H][W]
  const float2* maps = nullptr;
  const float* mask = nullptr;  // device, centred order
  int mask_is_lines = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 148;
  std::vector<float> mask_h;    // host copy (centred order)
  float* mask2s = nullptr;      // device: mask^2/(H W), shifted to plain FFT order
  LinesTables lines;
  Fft1D fH, fW;
  // non-Cartesian plans (Toeplitz embedding, Sec. 2.3.3): FFTs on the 2H x 2W grid and the
  // transformed PSF, psf_hat = FFT2(PSF) / (4 H W), complex64 [2H][2W] (plan-owned)
  int toep = 0;
  Fft1D fH2, fW2;
  float2* psf_hat = nullptr;
  // Bluestein tables of the generic normal operator's row passes (128 < W <= 256 with a radix
  // above 7, one map set; plan-owned, null otherwise): roots of the 512-point transforms | chirp
  // e^{-pi i n^2/W} [256] | chirp e^{+pi i n^2/W} [256] | the two convolution spectra [512]
  float2* blue = nullptr;
  // per-thread-index twiddle tables of the register-resident 512- and 256-point transforms
  // (plan-owned, null where no such transform is used)
  float2* twtab = nullptr;
  // P of the direct row passes of the generic normal operator (W = 8 P, P prime 17 .. 31, one map
  // set); 0 where they are not used
  int r8p = 0;
  int* status = nullptr;        // device status word (plan-owned)
  // bounded waits of the one-launch CG (sense_plan_set_wait_limit): polls of a per-slice
  // barrier before a CTA gives up, and arrivals added to every barrier (1 makes it unreachable)
  unsigned wait_polls = 1u << 22;
  unsigned wait_phantom = 0;
  int coop_set = 0;  // barrier-word set of the next one-launch CG solve (0 or 1, alternating)
  void* own = nullptr;          // plan-owned device allocation (tables + status)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  Workspace w;
};

// Process-wide launch accounting and per-kernel-class CUDA-event timing (profile.cu).
void prof_count(int n);

// Library-owned side streams, three per device (created on first use), for work inside one call
// that can run beside the caller's stream; events fork them from and join them back to it, so a
// call still completes in the caller's stream order (except where a call documents otherwise).
constexpr int kSideStreams = 3;
struct SideSet {
  cudaStream_t s[kSideStreams];
  cudaEvent_t ev;
};
int side_set(SideSet** out);
// `to` waits for the work issued so far on `from`
int stream_after(const SideSet& ss, cudaStream_t from, cudaStream_t to);
void prof_mark(const char* name, cudaStream_t s, bool stop);
inline void count_launch(sense_plan, int n = 1) { prof_count(n); }

// --------------------------------------------------------------- launchers
// Modes of the fused line-mask normal-operator kernel.
// NM_ADJ is the adjoint's row pass: x = sum_c conj(S_c) IDFT_W(T_c) from the sampled columns of
// the column-transformed k-space T (no phase A, no forward half of phase B).
// NM_CG2 is one pass of the single-reduction CG of the one-launch solve (see k_cg_lines).
enum NormalMode { NM_PLAIN = 0, NM_CG = 1, NM_RESID = 2, NM_ADJ = 3, NM_CG2 = 4 };

struct NormalLaunch {
  int mode = NM_PLAIN;
  const float2* x = nullptr;     // input (NM_CG: r)
  const float2* pold = nullptr;  // NM_CG: previous direction (NULL on iteration 0)
  float2* pout = nullptr;        // NM_CG: new direction written here
  float2* out = nullptr;
  const float2* rhs = nullptr;   // NM_RESID: out = rhs - S x
  float lam_host = 0.f;
  const double* lam_dev = nullptr;  // per-slice lambda [B] if non-NULL
  const double* beta = nullptr;     // NM_CG: [B]
  double* part = nullptr;        // [B][H] row partials: Re<x_eff, out> (NM_RESID: ||out||^2)
  int finalize = 0;              // 1: alpha = rr / pq; 2: rr = sum (+ rr_hist row)
  double* rr_hist_row = nullptr;
};

int launch_normal_lines(sense_plan p, const NormalLaunch& L);
// The region of a MoDL denoiser workspace that keeps an unrolled step's z = D(x_t).
float2* modl_zout(void* ws, int B, int H, int W);
// Every CG iteration in one cooperative launch (p->lines.coop): x, w.r, w.p, w.q, w.rr as left by
// the initial residual; rr_hist rows 1..iters written when non-NULL (without it the final
// residual and its norm are not formed: w.r and w.rr then hold those of the last iteration but one).
// rhs0: when not NULL the solve starts from x = 0, r = rhs0 (set in its first pass)
// lam: device FP64, lam_count = 1 (shared by the slices) or B (one per slice), read in place.
// rhs0b (with rhs0): the first pass stages r = rhs0 + lambda rhs0b; xlam: the last pass also
// writes lambda x there (both NULL when not wanted).
int launch_cg_lines(sense_plan p, float2* x, int iters, double* rr_hist, const float2* rhs0, const double* lam,
                    int lam_count, const float2* rhs0b, float2* xlam);
int build_lines_tables(sense_plan p);
void free_lines_tables(sense_plan p);

int build_fft1d(Fft1D& f, int L, std::vector<float2>& host_tw);
int generic_prepare(sense_plan p);
int launch_forward_generic(sense_plan p, const float2* x, float2* y);
int launch_adjoint_generic(sense_plan p, const float2* y, float2* x);
int launch_normal_generic(sense_plan p, const float2* x, float2* out, float lam_host,
                          const double* lam_dev);
int toeplitz_prepare(sense_plan p, const float2* psf);  // psf_hat from the PSF, kernel attributes
int launch_normal_toeplitz(sense_plan p, const float2* x, float2* out, float lam_host,
                           const double* lam_dev, double* dpart);
// True when launch_normal_toeplitz can also write the rows of Re<x, out> into dpart ([B][H][2]
// FP64: one slot per warp of a row, summed in slot order by the CG finalize).
bool toeplitz_fused_dot(sense_plan p);

int cg_run(sense_plan p, const float2* rhs, const float2* x0, float2* x, const double* lam,
           int lam_count, int iters, double* rr_hist);
// True when cg_run with x0 == NULL runs as one cooperative launch (the line-mask fused kernel).
bool cg_one_launch(sense_plan p, int iters);
// The one-launch solve from x0 = 0 of (A^H A + lambda I) x = rhs + lambda rhs_b, with lambda x also
// written to xlam when it is not NULL (the MoDL block's right-hand side and its reverse-mode
// scaling, fused into the first and last passes).  Only where cg_one_launch(p, iters).
int cg_run_one_launch(sense_plan p, const float2* rhs, const float2* rhs_b, float2* x, const double* lam,
                      int lam_count, int iters, double* rr_hist, float2* xlam);
int launch_dot_rows(sense_plan p, const float2* a, const float2* b, const float2* c,
                    double* out, int out_count, int accumulate);

// VarNet regulariser R(x) = sum_i K_i^T Phi_i'(K_i x) alone (varnet.cu): the VarNet kind of the
// denoiser calls.  Parameters in the 6,553-value stage layout (lambda unused).
size_t vn_denoiser_bytes(int B, int H, int W);
int vn_denoiser_forward(const float* prm, const void* x, void* out, void* ws, size_t ws_bytes, int B, int H,
                        int W, cudaStream_t st);
int vn_denoiser_backward(const float* prm, const void* x, const void* grad_out, void* grad_x, float* grad_prm,
                         void* ws, size_t ws_bytes, int B, int H, int W, cudaStream_t st);
