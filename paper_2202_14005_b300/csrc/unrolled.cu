// MoDL unrolled block (Sec. 2.3.2, Eq. 6) forward and reverse mode, the MSE
// training loss and Adam updates.
//
//   forward:  z = D_W(x_t);  x_{t+1} = S_lambda^{-1}(A^H y + lambda z)   (CG from 0)
//   backward: z recomputed from x_t (checkpointing, Sec. 2.2.4);
//             v = S_lambda^{-1} g (second CG);  grad_lambda += Re<v, z - x_{t+1}>;
//             grad_z = lambda v;  grad_x_t = (dD/dx)^H grad_z, grad_W += ...
//
// The loss is L = mean |x - x_gt|^2 with gradient 2 (x - x_gt) / n (complex
// convention of Sec. 2.2.2).  Adam follows Kingma and Ba; it consumes the
// accumulated gradient and clears it for the next step.
#include <cmath>

#include "plan.cuh"

namespace {

constexpr int kWarps = 8;

__global__ void k_rhs(size_t n2, const float4* b, const float4* z, const double* lam, float4* out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  const float l = (float)lam[0];
  const float4 u = b[i], v = z[i];
  out[i] = make_float4(fmaf(l, v.x, u.x), fmaf(l, v.y, u.y), fmaf(l, v.z, u.z), fmaf(l, v.w, u.w));
}

__global__ void k_scale(size_t n2, const float4* v, const double* lam, float4* out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  const float l = (float)lam[0];
  const float4 u = v[i];
  out[i] = make_float4(l * u.x, l * u.y, l * u.z, l * u.w);
}

// loss partials per image row, grad = 2 (x - gt) / n; last CTA sums in row order.
__global__ void __launch_bounds__(kWarps * 32) k_mse(int rows, int W, const float4* x, const float4* gt,
                                                     float4* grad, double inv_n, double* part,
                                                     double* loss, unsigned* counter) {
  const int row = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row < rows) {
    const size_t off = (size_t)row * W / 2;
    float s = 0.f;
    const float sc = (float)(2.0 * inv_n);
    for (int i = lane; i < W / 2; i += 32) {
      const float4 a = x[off + i], b = gt[off + i];
      const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
      s = fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, fmaf(d.w, d.w, s))));
      grad[off + i] = make_float4(sc * d.x, sc * d.y, sc * d.z, sc * d.w);
    }
    const double t = warp_sum_d((double)s);
    if (lane == 0) part[row] = t;
  }
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    double t = lane_strided_sum(part, rows, lane);
    t = warp_sum_d(t);
    if (lane == 0) {
      loss[0] = t * inv_n;
      *counter = 0u;
    }
  }
}

// Per-slice normalisation (the VarNet data scaling, Sec. 2.3.1): m_b = max |x_b| from per-row
// maxima (order-independent, so exact and reproducible); then x_b /= m_b and, if given,
// other_b /= m_b; scale[b] = 1 / m_b (1 for an all-zero slice).
__global__ void __launch_bounds__(kWarps * 32) k_row_absmax(int rows, int W, const float2* x, float* rmax) {
  const int row = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  float m = 0.f;
  for (int i = lane; i < W; i += 32) {
    const float2 v = x[(size_t)row * W + i];
    m = fmaxf(m, v.x * v.x + v.y * v.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) rmax[row] = m;
}

__global__ void k_scale_slices(int B, int H, int W, const float* rmax, float2* x, float2* other, float* scale) {
  __shared__ float s_inv;
  const int b = blockIdx.y;
  if (threadIdx.x < 32) {
    float m = 0.f;
    for (int h = threadIdx.x; h < H; h += 32) m = fmaxf(m, rmax[(size_t)b * H + h]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      const float inv = m > 0.f ? 1.f / sqrtf(m) : 1.f;
      s_inv = inv;
      if (blockIdx.x == 0 && scale) scale[b] = inv;
    }
  }
  __syncthreads();
  const float inv = s_inv;
  const size_t n = (size_t)H * W;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float2 v = x[(size_t)b * n + i];
    x[(size_t)b * n + i] = make_float2(v.x * inv, v.y * inv);
    if (other) {
      v = other[(size_t)b * n + i];
      other[(size_t)b * n + i] = make_float2(v.x * inv, v.y * inv);
    }
  }
}

template <typename T>
__global__ void k_adam(size_t n, T* p, T* g, T* m, T* v, T lr, T b1, T b2, T eps, T c1, T c2, T lo) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T gi = g[i];
  const T mi = b1 * m[i] + (T(1) - b1) * gi;
  const T vi = b2 * v[i] + (T(1) - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  T pi = p[i] - lr * (mi / c1) / (sqrt(vi / c2) + eps);
  if (pi < lo) pi = lo;
  p[i] = pi;
  g[i] = T(0);
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_step(sense_plan p, int kind, const void* weights, const double* lambda, const void* AHy,
               void* dn_ws, size_t dn_ws_bytes) {
  if (!p || !weights || !lambda || !AHy || !dn_ws) return SENSE_EINVAL_PTR;
  if (kind != SENSE_DENOISER_MODL) return SENSE_EUNSUPPORTED;  // VarNet stages return earlier
  if (p->S != 1) return SENSE_EUNSUPPORTED;                    // one image per slice
  if (!p->ws) return SENSE_EWORKSPACE;
  if (dn_ws_bytes < denoiser_workspace_bytes(kind, p->B, p->H, p->W)) return SENSE_EWORKSPACE;
  if (!al16(AHy) || ((uintptr_t)lambda & 7u)) return SENSE_EINVAL_PTR;
  return SENSE_OK;
}

}  // namespace

extern "C" {

int unrolled_step(sense_plan p, int kind, const float* weights, const double* lambda, const void* AHy,
                  const void* x_t, void* x_next, int cg_iters, void* dn_ws, size_t dn_ws_bytes) {
  if (kind == SENSE_DENOISER_VARNET)  // Eq. 5: lambda_t is part of the stage parameters, no CG
    return varnet_stage(p, weights, AHy, x_t, x_next, nullptr, dn_ws, dn_ws_bytes);
  if (int e = check_step(p, kind, weights, lambda, AHy, dn_ws, dn_ws_bytes)) return e;
  if (!x_t || !x_next || !al16(x_t) || !al16(x_next) || x_t == x_next) return SENSE_EINVAL_PTR;
  if (cg_iters < 0 || cg_iters > 100000) return SENSE_EINVAL_ARG;
  Workspace& w = p->w;
  const size_t n2 = (size_t)p->B * p->H * p->W / 2;
  // z lands in the denoiser workspace, next to the activations, for a backward that reuses them
  float2* z = modl_zout(dn_ws, p->B, p->H, p->W);
  if (int e = denoiser_forward(kind, weights, x_t, z, dn_ws, dn_ws_bytes, p->B, p->H, p->W, p->stream))
    return e;
  // rhs = A^H y + lambda z: formed by the one-launch solve's first pass where it applies
  if (cg_one_launch(p, cg_iters))
    return cg_run_one_launch(p, static_cast<const float2*>(AHy), z, static_cast<float2*>(x_next), lambda, 1,
                             cg_iters, nullptr, nullptr);
  prof_mark("unrolled_misc", p->stream, false);
  k_rhs<<<(unsigned)((n2 + 255) / 256), 256, 0, p->stream>>>(n2, static_cast<const float4*>(AHy),
                                                             reinterpret_cast<const float4*>(z), lambda,
                                                             reinterpret_cast<float4*>(w.t1));
  prof_mark("unrolled_misc", p->stream, true);
  count_launch(p);
  return cg_run(p, w.t1, nullptr, static_cast<float2*>(x_next), lambda, 1, cg_iters, nullptr);
}

int unrolled_step_backward_ex(sense_plan p, int kind, const float* weights, const double* lambda,
                              const void* AHy, const void* x_t, const void* x_next, const void* grad_next,
                              void* grad_t, float* grad_weights, double* grad_lambda, int cg_iters,
                              void* dn_ws, size_t dn_ws_bytes, int recompute) {
  if (kind == SENSE_DENOISER_VARNET)  // d/d lambda_t lands in grad_weights (stage layout)
    return varnet_stage_backward_ex(p, weights, AHy, x_t, nullptr, grad_next, grad_t, grad_weights, dn_ws,
                                    dn_ws_bytes, recompute);
  if (int e = check_step(p, kind, weights, lambda, AHy, dn_ws, dn_ws_bytes)) return e;
  if (!x_t || !x_next || !grad_next || !grad_t || !grad_weights || !grad_lambda || !al16(x_t) ||
      !al16(x_next) || !al16(grad_next) || !al16(grad_t) || grad_t == grad_next)
    return SENSE_EINVAL_PTR;
  if (cg_iters < 0 || cg_iters > 100000) return SENSE_EINVAL_ARG;
  Workspace& w = p->w;
  const size_t n2 = (size_t)p->B * p->H * p->W / 2;
  // z = D(x_t): recomputed (checkpointing), or as the forward step left it in dn_ws together with
  // the activations
  float2* z = modl_zout(dn_ws, p->B, p->H, p->W);
  if (recompute)
    if (int e = denoiser_forward(kind, weights, x_t, z, dn_ws, dn_ws_bytes, p->B, p->H, p->W, p->stream))
      return e;
  // v = S^{-1} g  and  grad_lambda += Re<v, z - x_next>;  grad_z = lambda v, written by the
  // one-launch solve's last pass where it applies
  const bool one = cg_one_launch(p, cg_iters);
  if (int e = one ? cg_run_one_launch(p, static_cast<const float2*>(grad_next), nullptr, w.t1, lambda, 1, cg_iters,
                                      nullptr, w.t0)
                  : cg_run(p, static_cast<const float2*>(grad_next), nullptr, w.t1, lambda, 1, cg_iters, nullptr))
    return e;
  if (int e = launch_dot_rows(p, w.t1, z, static_cast<const float2*>(x_next), grad_lambda, 1, 1))
    return e;
  if (!one) {
    prof_mark("unrolled_misc", p->stream, false);
    k_scale<<<(unsigned)((n2 + 255) / 256), 256, 0, p->stream>>>(n2, reinterpret_cast<const float4*>(w.t1),
                                                                 lambda, reinterpret_cast<float4*>(w.t0));
    prof_mark("unrolled_misc", p->stream, true);
    count_launch(p);
  }
  return denoiser_backward(kind, weights, x_t, w.t0, grad_t, grad_weights, dn_ws, dn_ws_bytes, p->B, p->H,
                           p->W, 0, p->stream);
}

int unrolled_step_backward(sense_plan p, int kind, const float* weights, const double* lambda,
                           const void* AHy, const void* x_t, const void* x_next, const void* grad_next,
                           void* grad_t, float* grad_weights, double* grad_lambda, int cg_iters,
                           void* dn_ws, size_t dn_ws_bytes) {
  return unrolled_step_backward_ex(p, kind, weights, lambda, AHy, x_t, x_next, grad_next, grad_t, grad_weights,
                                   grad_lambda, cg_iters, dn_ws, dn_ws_bytes, 1);
}

int sense_mse_loss(sense_plan p, const void* x, const void* gt, double* loss, void* grad) {
  if (!p || !x || !gt || !loss || !grad || !al16(x) || !al16(gt) || !al16(grad) || ((uintptr_t)loss & 7u))
    return SENSE_EINVAL_PTR;
  if (!p->ws) return SENSE_EWORKSPACE;
  const int rows = p->B * p->S * p->H;  // every map-set image of every slice
  const double inv_n = 1.0 / ((double)rows * p->W);
  prof_mark("unrolled_misc", p->stream, false);
  k_mse<<<(rows + kWarps - 1) / kWarps, kWarps * 32, 0, p->stream>>>(
      rows, p->W, static_cast<const float4*>(x), static_cast<const float4*>(gt), static_cast<float4*>(grad),
      inv_n, p->w.part, loss, p->w.counter);
  prof_mark("unrolled_misc", p->stream, true);
  count_launch(p);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int sense_normalize_max(sense_plan p, void* x, void* other, float* scale) {
  if (!p || !x || !al16(x) || (other && (!al16(other) || other == x)) || (scale && ((uintptr_t)scale & 3u)))
    return SENSE_EINVAL_PTR;
  if (!p->ws) return SENSE_EWORKSPACE;
  const int HS = p->S * p->H;  // a slice holds S map-set images
  const int rows = p->B * HS;
  float* rmax = reinterpret_cast<float*>(p->w.part);  // [B][S*H] scratch (the row-partial buffer)
  prof_mark("unrolled_misc", p->stream, false);
  k_row_absmax<<<(rows + kWarps - 1) / kWarps, kWarps * 32, 0, p->stream>>>(rows, p->W,
                                                                           static_cast<const float2*>(x), rmax);
  const int per = (int)(((size_t)HS * p->W + 255) / 256);
  k_scale_slices<<<dim3(min(per, 64), p->B), 256, 0, p->stream>>>(p->B, HS, p->W, rmax, static_cast<float2*>(x),
                                                                  static_cast<float2*>(other), scale);
  prof_mark("unrolled_misc", p->stream, true);
  prof_count(2);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int adam_update_f32(float* param, float* grad, float* m, float* v, size_t n, float lr, float beta1,
                    float beta2, float eps, int step, void* stream) {
  if (!param || !grad || !m || !v) return SENSE_EINVAL_PTR;
  if (step < 1 || !(lr >= 0.f)) return SENSE_EINVAL_ARG;
  const float c1 = (float)(1.0 - std::pow((double)beta1, step));
  const float c2 = (float)(1.0 - std::pow((double)beta2, step));
  prof_mark("unrolled_misc", static_cast<cudaStream_t>(stream), false);
  k_adam<float><<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, param, grad, m, v, lr, beta1, beta2, eps, c1, c2, -INFINITY);
  prof_mark("unrolled_misc", static_cast<cudaStream_t>(stream), true);
  prof_count(1);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int adam_update_f64(double* param, double* grad, double* m, double* v, size_t n, double lr, double beta1,
                    double beta2, double eps, int step, double lower, void* stream) {
  if (!param || !grad || !m || !v) return SENSE_EINVAL_PTR;
  if (step < 1 || !(lr >= 0.0)) return SENSE_EINVAL_ARG;
  const double c1 = 1.0 - std::pow(beta1, step), c2 = 1.0 - std::pow(beta2, step);
  prof_mark("unrolled_misc", static_cast<cudaStream_t>(stream), false);
  k_adam<double><<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, param, grad, m, v, lr, beta1, beta2, eps, c1, c2, lower);
  prof_mark("unrolled_misc", static_cast<cudaStream_t>(stream), true);
  prof_count(1);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

}  // extern "C"
