// C ABI of libsense: plan life cycle, argument checks, workspace carving and
// dispatch to the kernels.  The contract of each call is in include/sense.h.
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "plan.cuh"

namespace {

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
size_t up256(size_t n) { return (n + 255) & ~(size_t)255; }

struct WsLayout {
  size_t T, r, p, q, t0, t1, wv, sv, part, part2, rr, alpha, beta, lam, counter, total;
};

WsLayout ws_layout(const sense_plan p) {
  WsLayout L;
  const size_t plane = (size_t)p->B * p->H * p->W * sizeof(float2);
  const size_t img = plane * p->S;  // images [B][S][H][W]
  size_t o = 0;
  L.T = o; o += up256(plane * p->C * (p->toep ? 2 : 1));  // Toeplitz plans: rows of length 2W
  L.r = o; o += up256(img);
  L.p = o; o += up256(img);
  L.q = o; o += up256(img);
  L.t0 = o; o += up256(img);
  L.t1 = o; o += up256(img);
  L.wv = o; o += up256(img);
  L.sv = o; o += up256(img);
  L.part = o; o += up256((size_t)p->B * p->S * p->H * sizeof(double));
  L.part2 = o; o += up256(4 * (size_t)p->B * p->S * p->H * sizeof(double));  // one-launch CG: 4 sets
  L.rr = o; o += up256(p->B * sizeof(double));
  L.alpha = o; o += up256(p->B * sizeof(double));
  L.beta = o; o += up256(p->B * sizeof(double));
  L.lam = o; o += up256(p->B * sizeof(double));
  L.counter = o; o += 12288;  // counters, the one-launch CG scalars and two sets of barrier words
  L.total = o;
  return L;
}

int need_ws(sense_plan p) { return p->ws ? SENSE_OK : SENSE_EWORKSPACE; }

}  // namespace

extern "C" {

const char* sense_strerror(int code) {
  switch (code) {
    case SENSE_OK: return "ok";
    case SENSE_EINVAL_SHAPE: return "invalid shape (sizes must be positive, H and W even)";
    case SENSE_EINVAL_PTR: return "NULL, aliased or misaligned pointer";
    case SENSE_EINVAL_LAMBDA: return "invalid lambda (must be finite and >= 0)";
    case SENSE_EUNSUPPORTED: return "unsupported size (prime factor above 31, or too large)";
    case SENSE_ECUDA: return "CUDA runtime error";
    case SENSE_EWORKSPACE: return "workspace missing or too small";
    case SENSE_EINVAL_ARG: return "invalid argument";
    case SENSE_ETOO_LARGE: return "problem exceeds the fixed scratch of the no-allocation entry point";
    default: return "unknown error code";
  }
}

int sense_plan_create(sense_plan* out, int B, int C, int H, int W, const void* maps,
                      const float* mask, int mask_is_lines, void* stream) {
  return sense_plan_create_sets(out, B, 1, C, H, W, maps, mask, mask_is_lines, stream);
}

int sense_plan_create_sets(sense_plan* out, int B, int S, int C, int H, int W, const void* maps,
                           const float* mask, int mask_is_lines, void* stream) {
  if (!out) return SENSE_EINVAL_PTR;
  *out = nullptr;
  if (B <= 0 || S <= 0 || C <= 0 || H <= 0 || W <= 0 || (H & 1) || (W & 1)) return SENSE_EINVAL_SHAPE;
  if (S > 8) return SENSE_EUNSUPPORTED;
  if ((long long)B * S * C * H * W > (1ll << 34)) return SENSE_EUNSUPPORTED;
  if (!maps || !mask || !aligned16(maps) || !aligned16(mask)) return SENSE_EINVAL_PTR;
  if (mask_is_lines != 0 && mask_is_lines != 1) return SENSE_EINVAL_ARG;
  std::vector<float2> twH, twW;
  Fft1D fH, fW;
  if (int e = build_fft1d(fH, H, twH)) return e;
  if (int e = build_fft1d(fW, W, twW)) return e;
  sense_plan p = new (std::nothrow) sense_plan_s();
  if (!p) return SENSE_ECUDA;
  p->B = B; p->C = C; p->H = H; p->W = W; p->S = S;
  p->maps = static_cast<const float2*>(maps);
  p->mask = mask;
  p->mask_is_lines = mask_is_lines;
  p->stream = static_cast<cudaStream_t>(stream);
  p->fH = fH;
  p->fW = fW;
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    delete p;
    return SENSE_ECUDA;
  }
  // host copy of the mask (centred order) and the shifted mask^2/(HW) table
  const size_t mn = mask_is_lines ? (size_t)W : (size_t)H * W;
  p->mask_h.resize(mn);
  if (cudaMemcpyAsync(p->mask_h.data(), mask, mn * sizeof(float), cudaMemcpyDeviceToHost,
                      p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    delete p;
    return SENSE_ECUDA;
  }
  std::vector<float> m2s(mn);
  const double sc = 1.0 / ((double)H * W);
  if (mask_is_lines) {
    for (int k = 0; k < W; ++k) {
      const double m = p->mask_h[(k + W / 2) % W];
      m2s[k] = (float)(m * m * sc);
    }
  } else {
    for (int kh = 0; kh < H; ++kh)
      for (int kw = 0; kw < W; ++kw) {
        const double m = p->mask_h[(size_t)((kh + H / 2) % H) * W + (kw + W / 2) % W];
        m2s[(size_t)kh * W + kw] = (float)(m * m * sc);
      }
  }
  // plan-owned device block: status word | twH | twW | mask2s
  const size_t o_tH = 256, o_tW = o_tH + up256(H * sizeof(float2)),
               o_m = o_tW + up256(W * sizeof(float2)), tot = o_m + up256(mn * sizeof(float));
  char* d = nullptr;
  if (cudaMalloc(&d, tot) != cudaSuccess) {
    delete p;
    return SENSE_ECUDA;
  }
  p->own = d;
  p->status = reinterpret_cast<int*>(d);
  p->fH.tw = reinterpret_cast<float2*>(d + o_tH);
  p->fW.tw = reinterpret_cast<float2*>(d + o_tW);
  p->mask2s = reinterpret_cast<float*>(d + o_m);
  if (cudaMemset(d, 0, 256) != cudaSuccess ||
      cudaMemcpy(p->fH.tw, twH.data(), H * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->fW.tw, twW.data(), W * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->mask2s, m2s.data(), mn * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    sense_plan_destroy(p);
    return SENSE_ECUDA;
  }
  int err = generic_prepare(p);
  if (!err) err = build_lines_tables(p);  // fused line-mask kernel where one is compiled
  if (err) {
    sense_plan_destroy(p);
    return err;
  }
  *out = p;
  return SENSE_OK;
}

int sense_plan_create_toeplitz(sense_plan* out, int B, int C, int H, int W, const void* maps, const void* psf,
                               void* stream) {
  if (!out) return SENSE_EINVAL_PTR;
  *out = nullptr;
  if (B <= 0 || C <= 0 || H <= 0 || W <= 0 || (H & 1) || (W & 1)) return SENSE_EINVAL_SHAPE;
  if ((long long)B * C * H * W > (1ll << 33)) return SENSE_EUNSUPPORTED;
  if (!maps || !psf || !aligned16(maps) || !aligned16(psf)) return SENSE_EINVAL_PTR;
  std::vector<float2> twH, twW, twH2, twW2;
  Fft1D fH, fW, fH2, fW2;
  if (int e = build_fft1d(fH, H, twH)) return e;
  if (int e = build_fft1d(fW, W, twW)) return e;
  if (int e = build_fft1d(fH2, 2 * H, twH2)) return e;
  if (int e = build_fft1d(fW2, 2 * W, twW2)) return e;
  sense_plan p = new (std::nothrow) sense_plan_s();
  if (!p) return SENSE_ECUDA;
  p->B = B; p->C = C; p->H = H; p->W = W; p->S = 1;
  p->toep = 1;
  p->maps = static_cast<const float2*>(maps);
  p->stream = static_cast<cudaStream_t>(stream);
  p->fH = fH; p->fW = fW; p->fH2 = fH2; p->fW2 = fW2;
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    delete p;
    return SENSE_ECUDA;
  }
  // plan-owned device block: status word | twH2 | twW2 | psf_hat [2H][2W]
  const size_t o_tH = 256, o_tW = o_tH + up256(2 * H * sizeof(float2)),
               o_p = o_tW + up256(2 * W * sizeof(float2)), tot = o_p + up256((size_t)4 * H * W * sizeof(float2));
  char* d = nullptr;
  if (cudaMalloc(&d, tot) != cudaSuccess) {
    delete p;
    return SENSE_ECUDA;
  }
  p->own = d;
  p->status = reinterpret_cast<int*>(d);
  p->fH2.tw = reinterpret_cast<float2*>(d + o_tH);
  p->fW2.tw = reinterpret_cast<float2*>(d + o_tW);
  p->psf_hat = reinterpret_cast<float2*>(d + o_p);
  if (cudaMemset(d, 0, 256) != cudaSuccess ||
      cudaMemcpy(p->fH2.tw, twH2.data(), 2 * H * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->fW2.tw, twW2.data(), 2 * W * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
    sense_plan_destroy(p);
    return SENSE_ECUDA;
  }
  if (int e = toeplitz_prepare(p, static_cast<const float2*>(psf))) {
    sense_plan_destroy(p);
    return e;
  }
  *out = p;
  return SENSE_OK;
}

int sense_plan_destroy(sense_plan p) {
  if (!p) return SENSE_EINVAL_PTR;
  free_lines_tables(p);
  if (p->own) cudaFree(p->own);
  if (p->blue) cudaFree(p->blue);
  if (p->twtab) cudaFree(p->twtab);
  delete p;
  return SENSE_OK;
}

int sense_plan_set_stream(sense_plan p, void* stream) {
  if (!p) return SENSE_EINVAL_PTR;
  p->stream = static_cast<cudaStream_t>(stream);
  return SENSE_OK;
}

int sense_plan_workspace_bytes(sense_plan p, size_t* bytes) {
  if (!p || !bytes) return SENSE_EINVAL_PTR;
  *bytes = ws_layout(p).total;
  return SENSE_OK;
}

int sense_plan_set_workspace(sense_plan p, void* ws, size_t bytes) {
  if (!p || !ws || ((uintptr_t)ws & 255u)) return SENSE_EINVAL_PTR;
  const WsLayout L = ws_layout(p);
  if (bytes < L.total) return SENSE_EWORKSPACE;
  char* b = static_cast<char*>(ws);
  p->ws = ws;
  p->ws_bytes = bytes;
  Workspace& w = p->w;
  w.T = reinterpret_cast<float2*>(b + L.T);
  w.r = reinterpret_cast<float2*>(b + L.r);
  w.p = reinterpret_cast<float2*>(b + L.p);
  w.q = reinterpret_cast<float2*>(b + L.q);
  w.t0 = reinterpret_cast<float2*>(b + L.t0);
  w.t1 = reinterpret_cast<float2*>(b + L.t1);
  w.wv = reinterpret_cast<float2*>(b + L.wv);
  w.sv = reinterpret_cast<float2*>(b + L.sv);
  w.part = reinterpret_cast<double*>(b + L.part);
  w.part2 = reinterpret_cast<double*>(b + L.part2);
  w.rr = reinterpret_cast<double*>(b + L.rr);
  w.alpha = reinterpret_cast<double*>(b + L.alpha);
  w.beta = reinterpret_cast<double*>(b + L.beta);
  w.lam = reinterpret_cast<double*>(b + L.lam);
  w.counter = reinterpret_cast<unsigned*>(b + L.counter);
  return cudaMemsetAsync(w.counter, 0, 12288, p->stream) == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int sense_forward(sense_plan p, const void* x, void* y) {
  if (!p || !x || !y || !aligned16(x) || !aligned16(y) || x == y) return SENSE_EINVAL_PTR;
  if (p->toep) return SENSE_EUNSUPPORTED;  // non-Cartesian plans hold the normal operator only
  return launch_forward_generic(p, static_cast<const float2*>(x), static_cast<float2*>(y));
}

int sense_adjoint(sense_plan p, const void* y, void* x) {
  if (!p || !x || !y || !aligned16(x) || !aligned16(y) || x == y) return SENSE_EINVAL_PTR;
  if (p->toep) return SENSE_EUNSUPPORTED;
  if (int e = need_ws(p)) return e;
  return launch_adjoint_generic(p, static_cast<const float2*>(y), static_cast<float2*>(x));
}

int sense_normal(sense_plan p, const void* x, void* out, float lambda) {
  if (!p || !x || !out || !aligned16(x) || !aligned16(out) || x == out) return SENSE_EINVAL_PTR;
  if (!std::isfinite(lambda) || lambda < 0.f) return SENSE_EINVAL_LAMBDA;
  if (p->lines.ok) {
    NormalLaunch L;
    L.mode = NM_PLAIN;
    L.x = static_cast<const float2*>(x);
    L.out = static_cast<float2*>(out);
    L.lam_host = lambda;
    return launch_normal_lines(p, L);
  }
  if (int e = need_ws(p)) return e;
  return launch_normal_generic(p, static_cast<const float2*>(x), static_cast<float2*>(out), lambda,
                               nullptr);
}

int cg_dc_solve(sense_plan p, const void* rhs, const void* x0, void* x, const double* lambda,
                int lambda_count, int iters, double* rr_hist) {
  if (!p || !rhs || !x || !lambda || !aligned16(rhs) || !aligned16(x) || (x0 && !aligned16(x0)) ||
      rhs == x)
    return SENSE_EINVAL_PTR;
  if (((uintptr_t)lambda & 7u) || (rr_hist && ((uintptr_t)rr_hist & 7u))) return SENSE_EINVAL_PTR;
  if (lambda_count != 1 && lambda_count != p->B) return SENSE_EINVAL_ARG;
  if (iters < 0 || iters > 100000) return SENSE_EINVAL_ARG;
  if (int e = need_ws(p)) return e;
  return cg_run(p, static_cast<const float2*>(rhs), static_cast<const float2*>(x0),
                static_cast<float2*>(x), lambda, lambda_count, iters, rr_hist);
}

int cg_dc_solve_backward(sense_plan p, const void* grad_x, const void* x, const void* z,
                         const double* lambda, int lambda_count, int iters, void* grad_rhs,
                         double* grad_lambda) {
  if (!p || !grad_x || !x || !lambda || !grad_rhs || !aligned16(grad_x) || !aligned16(x) ||
      (z && !aligned16(z)) || !aligned16(grad_rhs) || grad_rhs == grad_x)
    return SENSE_EINVAL_PTR;
  if (((uintptr_t)lambda & 7u) || (grad_lambda && ((uintptr_t)grad_lambda & 7u)))
    return SENSE_EINVAL_PTR;
  if (lambda_count != 1 && lambda_count != p->B) return SENSE_EINVAL_ARG;
  if (iters < 0 || iters > 100000) return SENSE_EINVAL_ARG;
  if (int e = need_ws(p)) return e;
  float2* v = static_cast<float2*>(grad_rhs);
  if (int e = cg_run(p, static_cast<const float2*>(grad_x), nullptr, v, lambda, lambda_count, iters,
                     nullptr))
    return e;
  if (grad_lambda)
    return launch_dot_rows(p, v, static_cast<const float2*>(z), static_cast<const float2*>(x),
                           grad_lambda, lambda_count, 0);
  return SENSE_OK;
}

int sense_plan_set_wait_limit(sense_plan p, unsigned polls, int unreachable) {
  if (!p) return SENSE_EINVAL_PTR;
  if (unreachable != 0 && unreachable != 1) return SENSE_EINVAL_ARG;
  p->wait_polls = polls ? polls : (1u << 22);
  p->wait_phantom = (unsigned)unreachable;
  return SENSE_OK;
}

int sense_get_status(sense_plan p, int* device_status) {
  if (!p || !device_status) return SENSE_EINVAL_PTR;
  int v = 0;
  if (cudaMemcpyAsync(&v, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess ||
      cudaMemsetAsync(p->status, 0, sizeof(int), p->stream) != cudaSuccess)
    return SENSE_ECUDA;
  *device_status = v;
  return SENSE_OK;
}

}  // extern "C"
