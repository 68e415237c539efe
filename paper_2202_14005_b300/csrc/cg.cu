// Conjugate gradient on S_lambda = A^H A + lambda I, independently per slice
// (Sec. 2.3.2, MoDL data consistency), and the inner products of its
// derivative.  Vectors are FP32 complex; every inner product is formed from
// FP32 products summed per lane over a few elements, then carried in FP64:
// per-row partials, reduced per slice in a fixed order by the last CTA of each
// launch (no floating-point atomics: results are bitwise reproducible).
// alpha and beta are FP64 and stay on the device: the host never waits.
//
// Per iteration i (Hestenes-Stiefel):
//   N kernel: p = r + beta p (p = r at i = 0); q = S p; part = Re<p, q>;
//             last CTA: alpha = ||r||^2 / Re<p, q>
//   U kernel: x += alpha p; r -= alpha q; part = ||r||^2;
//             last CTA: beta = ||r_new||^2 / ||r||^2, ||r||^2 <- ||r_new||^2
// A slice with ||r||^2 == 0 gets alpha = beta = 0 (frozen).  Re<p, q> <= 0
// with ||r||^2 > 0 sets SENSE_STATUS_CG_BREAKDOWN; non-finite scalars set
// SENSE_STATUS_NONFINITE; both leave alpha = 0 so the iteration is a no-op.
#include <cmath>

#include "plan.cuh"

namespace {

constexpr int kWarps = 8;

enum Fin { FIN_NONE = 0, FIN_RR0 = 1, FIN_ALPHA = 2, FIN_RRNEW = 3, FIN_GLAM = 4 };

struct RowArgs {
  int B, H, W;
  const float2* a;   // roles documented at each kernel
  const float2* b;
  const float2* c;
  float2* o1;
  float2* o2;
  double* part;      // [B][H]
  int fin;
  double* rr;
  double* alpha;
  double* beta;
  double* hist;      // rr_hist row [B] or NULL
  double* gout;      // FIN_GLAM output
  int gcount;        // 1 or B
  int gacc;          // FIN_GLAM: add to gout instead of overwriting
  unsigned* counter;
  int* status;
};

// Per slice: the fixed-order sum of its row partials (a warp per slice, warp, warp + nwarps, ...),
// then, one thread per slice, the scalar update: the FP64 divisions of all slices run side by
// side instead of one after another in each warp's lane 0.  kFinChunk slices per round (their
// sums are held in shared memory between the two steps).
constexpr int kFinChunk = 256;
__device__ void finalize_slice(const RowArgs& a, int b, double s);

__device__ void finalize(const RowArgs& a) {
  __shared__ double s_sum[kFinChunk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int b0 = 0; b0 < a.B; b0 += kFinChunk) {
    const int nb = min(kFinChunk, a.B - b0);
    for (int i = warp; i < nb; i += nwarps) {
      const double s = warp_sum_d(lane_strided_sum(a.part + (size_t)(b0 + i) * a.H, a.H, lane));
      if (lane == 0) s_sum[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) finalize_slice(a, b0 + i, s_sum[i]);
    __syncthreads();
  }
  if (a.fin == FIN_GLAM && a.gcount != a.B) {
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int b = 0; b < a.B; ++b) t += a.alpha[b];
      a.gout[0] = a.gacc ? a.gout[0] + t : t;
    }
  }
}

__device__ void finalize_slice(const RowArgs& a, int b, double s) {
  {
    if (a.fin == FIN_RR0) {
      if (!isfinite(s)) set_status(a.status, SENSE_DEVST_NONFINITE);
      a.rr[b] = s;
      if (a.hist) a.hist[b] = s;
    } else if (a.fin == FIN_ALPHA) {
      const double rr = __ldcg(a.rr + b);
      double al = 0.0;
      if (!isfinite(s) || !isfinite(rr)) set_status(a.status, SENSE_DEVST_NONFINITE);
      else if (rr > 0.0) {
        if (s > 0.0) al = rr / s;
        else set_status(a.status, SENSE_DEVST_CG_BREAKDOWN);
      }
      a.alpha[b] = al;
    } else if (a.fin == FIN_RRNEW) {
      const double ro = __ldcg(a.rr + b);
      if (!isfinite(s)) set_status(a.status, SENSE_DEVST_NONFINITE);
      a.beta[b] = (ro > 0.0 && isfinite(s)) ? s / ro : 0.0;
      a.rr[b] = s;
      if (a.hist) a.hist[b] = s;
    } else if (a.fin == FIN_GLAM) {
      if (a.gcount == a.B) a.gout[b] = a.gacc ? a.gout[b] + s : s;
      else a.alpha[b] = s;  // per-slice scratch, summed in slice order by finalize
    }
  }
}

__device__ void last_block(const RowArgs& a) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(a.counter, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    finalize(a);
    __syncthreads();
    if (threadIdx.x == 0) *a.counter = 0u;
  }
}

// Two warps per image row (four rows per 256-thread CTA and pass); elements are
// taken two at a time (float4 = 2 complex).  Each warp reduces its FP32 lane
// sums in FP64; the two warp sums of a row are added in warp order.  A CTA
// takes the groups of four rows blockIdx.x, blockIdx.x + gridDim.x, ... (a
// grid of kCtasPerSm CTAs per SM): fewer CTAs, and so fewer fences and
// counter increments of the last-CTA reduction.
constexpr int kRowsPerCta = kWarps / 2;
constexpr int kCtasPerSm = 4;

__device__ __forceinline__ void row_partial(const RowArgs& a, int row, bool rv, float part) {
  __shared__ double s_w[kWarps];
  const double d = warp_sum_d((double)part);
  const int warp = threadIdx.x >> 5;
  __syncthreads();  // the previous group's sums have been read
  if ((threadIdx.x & 31) == 0) s_w[warp] = d;
  __syncthreads();
  if (rv && a.part && (threadIdx.x & 63) == 0) a.part[row] = s_w[warp] + s_w[warp + 1];
}

#define ROW_LOOP_BEGIN                                                    \
  for (int rbase = blockIdx.x * kRowsPerCta; rbase < a.B * a.H;           \
       rbase += gridDim.x * kRowsPerCta) {                                \
  const int row = rbase + (threadIdx.x >> 6);                             \
  const int lt = threadIdx.x & 63;                                        \
  const bool rv = row < a.B * a.H;                                        \
  float part = 0.f;                                                       \
  if (rv) {                                                               \
    const int b = row / a.H;                                              \
    (void)b;                                                              \
    const size_t off = (size_t)row * a.W / 2;                             \
    for (int i = lt; i < a.W / 2; i += 64) {
#define ROW_LOOP_END                                                      \
    }                                                                     \
  }                                                                       \
  row_partial(a, row, rv, part);                                          \
  }

__device__ __forceinline__ float nrm2(float4 v) {
  return fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, v.w * v.w)));
}
__device__ __forceinline__ float redot(float4 u, float4 v) {  // Re<u, v> over two complex
  return fmaf(u.x, v.x, fmaf(u.y, v.y, fmaf(u.z, v.z, u.w * v.w)));
}

// r (o1) = rhs (a), x (o2) = 0, part = ||r||^2
__global__ void __launch_bounds__(kWarps * 32) k_cg_init(const RowArgs a) {
  ROW_LOOP_BEGIN
  const float4 r = reinterpret_cast<const float4*>(a.a)[off + i];
  reinterpret_cast<float4*>(a.o1)[off + i] = r;
  reinterpret_cast<float4*>(a.o2)[off + i] = make_float4(0.f, 0.f, 0.f, 0.f);
  part += nrm2(r);
  ROW_LOOP_END
  if (a.fin) last_block(a);
}

// x (o1) += alpha p (a); r (o2) -= alpha q (b); part = ||r||^2
__global__ void __launch_bounds__(kWarps * 32) k_cg_update(const RowArgs a) {
  ROW_LOOP_BEGIN
  const float al = (float)a.alpha[b];
  const float4 p = reinterpret_cast<const float4*>(a.a)[off + i];
  const float4 q = reinterpret_cast<const float4*>(a.b)[off + i];
  float4 x = reinterpret_cast<float4*>(a.o1)[off + i];
  float4 r = reinterpret_cast<float4*>(a.o2)[off + i];
  x.x = fmaf(al, p.x, x.x); x.y = fmaf(al, p.y, x.y); x.z = fmaf(al, p.z, x.z); x.w = fmaf(al, p.w, x.w);
  r.x = fmaf(-al, q.x, r.x); r.y = fmaf(-al, q.y, r.y); r.z = fmaf(-al, q.z, r.z); r.w = fmaf(-al, q.w, r.w);
  reinterpret_cast<float4*>(a.o1)[off + i] = x;
  reinterpret_cast<float4*>(a.o2)[off + i] = r;
  part += nrm2(r);
  ROW_LOOP_END
  if (a.fin) last_block(a);
}

// p (o1) = r (a) + beta p (o1), or p = r when beta == NULL
__global__ void __launch_bounds__(kWarps * 32) k_cg_p(const RowArgs a) {
  ROW_LOOP_BEGIN
  const float4 r = reinterpret_cast<const float4*>(a.a)[off + i];
  float4 v = r;
  if (a.beta) {
    const float be = (float)a.beta[b];
    const float4 po = reinterpret_cast<float4*>(a.o1)[off + i];
    v.x = fmaf(be, po.x, r.x); v.y = fmaf(be, po.y, r.y); v.z = fmaf(be, po.z, r.z); v.w = fmaf(be, po.w, r.w);
  }
  reinterpret_cast<float4*>(a.o1)[off + i] = v;
  ROW_LOOP_END
}

// part = Re<a, b - c>  (b or c may be NULL, standing for zero)
__global__ void __launch_bounds__(kWarps * 32) k_dot(const RowArgs a) {
  ROW_LOOP_BEGIN
  const float4 u = reinterpret_cast<const float4*>(a.a)[off + i];
  float4 v = a.b ? reinterpret_cast<const float4*>(a.b)[off + i] : make_float4(0.f, 0.f, 0.f, 0.f);
  if (a.c) {
    const float4 w = reinterpret_cast<const float4*>(a.c)[off + i];
    v.x -= w.x; v.y -= w.y; v.z -= w.z; v.w -= w.w;
  }
  part += redot(u, v);
  ROW_LOOP_END
  if (a.fin) last_block(a);
}

// r (o1) = rhs (a) - r (o1); part = ||r||^2
__global__ void __launch_bounds__(kWarps * 32) k_resid(const RowArgs a) {
  ROW_LOOP_BEGIN
  const float4 bv = reinterpret_cast<const float4*>(a.a)[off + i];
  float4 r = reinterpret_cast<float4*>(a.o1)[off + i];
  r.x = bv.x - r.x; r.y = bv.y - r.y; r.z = bv.z - r.z; r.w = bv.w - r.w;
  reinterpret_cast<float4*>(a.o1)[off + i] = r;
  part += nrm2(r);
  ROW_LOOP_END
  if (a.fin) last_block(a);
}

// The per-slice reductions alone, over row partials another kernel wrote (one CTA).
__global__ void __launch_bounds__(256) k_cg_fin(const RowArgs a) { finalize(a); }

__global__ void k_lam_expand(int B, const double* lam, int count, double* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) out[b] = lam[count == 1 ? 0 : b];
}

RowArgs base_args(sense_plan p) {
  RowArgs a;
  a.B = p->B; a.H = p->S * p->H; a.W = p->W;  // [B][S][H][W] = [B][S*H][W] rows
  a.a = a.b = a.c = nullptr;
  a.o1 = a.o2 = nullptr;
  a.part = p->w.part;
  a.fin = FIN_NONE;
  a.rr = p->w.rr; a.alpha = p->w.alpha; a.beta = p->w.beta;
  a.hist = nullptr; a.gout = nullptr; a.gcount = 1; a.gacc = 0;
  a.counter = p->w.counter; a.status = p->status;
  return a;
}

int grid_rows(sense_plan p) {
  const int groups = (p->B * p->S * p->H + kRowsPerCta - 1) / kRowsPerCta;
  return groups < kCtasPerSm * p->num_sms ? groups : kCtasPerSm * p->num_sms;
}

}  // namespace

bool cg_one_launch(sense_plan p, int iters) { return p->lines.ok && p->lines.coop && iters > 0; }

int cg_run_one_launch(sense_plan p, const float2* rhs, const float2* rhs_b, float2* x, const double* lam,
                      int lam_count, int iters, double* rr_hist, float2* xlam) {
  if (!cg_one_launch(p, iters)) return SENSE_EUNSUPPORTED;
  return launch_cg_lines(p, x, iters, rr_hist, rhs, lam, lam_count, rhs_b, xlam);
}

int cg_run(sense_plan p, const float2* rhs, const float2* x0, float2* x, const double* lam,
           int lam_count, int iters, double* rr_hist) {
  Workspace& w = p->w;
  const int gr = grid_rows(p);
  const int B = p->B;
  // the one-launch solve reads lambda in place; the other paths take one value per slice
  const bool coop = p->lines.ok && p->lines.coop && iters > 0;
  if (!coop || x0) {
    prof_mark("cg_vec", p->stream, false);
    k_lam_expand<<<(B + 127) / 128, 128, 0, p->stream>>>(B, lam, lam_count, w.lam);
    prof_mark("cg_vec", p->stream, true);
    count_launch(p);
  }
  // ---- initial residual
  if (x0) {
    if (x0 != x &&
        cudaMemcpyAsync(x, x0, (size_t)B * p->S * p->H * p->W * sizeof(float2), cudaMemcpyDeviceToDevice,
                        p->stream) != cudaSuccess)
      return SENSE_ECUDA;
    if (p->lines.ok) {
      NormalLaunch L;
      L.mode = NM_RESID; L.x = x; L.out = w.r; L.rhs = rhs; L.lam_dev = w.lam;
      L.part = w.part; L.finalize = 2; L.rr_hist_row = rr_hist;
      if (int e = launch_normal_lines(p, L)) return e;
    } else {
      if (int e = launch_normal_generic(p, x, w.r, 0.f, w.lam)) return e;
      RowArgs a = base_args(p);
      a.a = rhs; a.o1 = w.r; a.fin = FIN_RR0; a.hist = rr_hist;
      prof_mark("cg_vec", p->stream, false);
      k_resid<<<gr, kWarps * 32, 0, p->stream>>>(a);
      prof_mark("cg_vec", p->stream, true);
      count_launch(p);
    }
  } else if (coop) {
    // x = 0, r = rhs and ||r||^2 in the first pass of the one-launch solve
    return launch_cg_lines(p, x, iters, rr_hist, rhs, lam, lam_count, nullptr, nullptr);
  } else {
    RowArgs a = base_args(p);
    a.a = rhs; a.o1 = w.r; a.o2 = x; a.fin = FIN_RR0; a.hist = rr_hist;
    prof_mark("cg_vec", p->stream, false);
    k_cg_init<<<gr, kWarps * 32, 0, p->stream>>>(a);
    prof_mark("cg_vec", p->stream, true);
    count_launch(p);
  }
  // ---- iterations: all of them in one cooperative launch where the fused kernel applies
  if (coop) return launch_cg_lines(p, x, iters, rr_hist, nullptr, lam, lam_count, nullptr, nullptr);
  for (int it = 0; it < iters; ++it) {
    double* hist = rr_hist ? rr_hist + (size_t)(it + 1) * B : nullptr;
    if (p->lines.ok) {
      NormalLaunch L;
      L.mode = NM_CG; L.x = w.r; L.pold = it ? w.p : nullptr; L.pout = w.p; L.out = w.q;
      L.lam_dev = w.lam; L.beta = w.beta; L.part = w.part; L.finalize = 1;
      if (int e = launch_normal_lines(p, L)) return e;
    } else {
      RowArgs a = base_args(p);
      a.a = w.r; a.o1 = w.p; a.beta = it ? w.beta : nullptr;
      prof_mark("cg_vec", p->stream, false);
      k_cg_p<<<gr, kWarps * 32, 0, p->stream>>>(a);
      prof_mark("cg_vec", p->stream, true);
      count_launch(p);
      RowArgs d = base_args(p);
      d.a = w.p; d.b = w.q; d.fin = FIN_ALPHA;
      if (toeplitz_fused_dot(p)) {
        // the operator's inverse row pass writes the rows of Re<p, q> (two slots per row)
        if (int e = launch_normal_toeplitz(p, w.p, w.q, 0.f, w.lam, w.part2)) return e;
        d.part = w.part2;
        d.H = 2 * p->S * p->H;
        prof_mark("cg_vec", p->stream, false);
        k_cg_fin<<<1, 256, 0, p->stream>>>(d);
        prof_mark("cg_vec", p->stream, true);
      } else {
        if (int e = launch_normal_generic(p, w.p, w.q, 0.f, w.lam)) return e;
        prof_mark("cg_vec", p->stream, false);
        k_dot<<<gr, kWarps * 32, 0, p->stream>>>(d);
        prof_mark("cg_vec", p->stream, true);
      }
      count_launch(p);
    }
    RowArgs u = base_args(p);
    u.a = w.p; u.b = w.q; u.o1 = x; u.o2 = w.r; u.fin = FIN_RRNEW; u.hist = hist;
    prof_mark("cg_vec", p->stream, false);
    k_cg_update<<<gr, kWarps * 32, 0, p->stream>>>(u);
    prof_mark("cg_vec", p->stream, true);
    count_launch(p);
  }
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

// out[count] (=, or += when accumulate) sum Re<a, b - c> per slice (count == B) or over all
// slices (count == 1).
int launch_dot_rows(sense_plan p, const float2* a_, const float2* b_, const float2* c_, double* out,
                    int out_count, int accumulate) {
  RowArgs a = base_args(p);
  a.a = a_; a.b = b_; a.c = c_; a.fin = FIN_GLAM; a.gout = out; a.gcount = out_count;
  a.gacc = accumulate;
  prof_mark("cg_vec", p->stream, false);
  k_dot<<<grid_rows(p), kWarps * 32, 0, p->stream>>>(a);
  prof_mark("cg_vec", p->stream, true);
  count_launch(p);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}
