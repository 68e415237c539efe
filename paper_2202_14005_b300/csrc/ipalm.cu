// iPALM update of the VarNet stage parameters with the filter constraints (Sec. 2.3.1 trains the
// VarNet with iPALM, the inertial proximal alternating linearised minimisation of Pock and
// Sabach).  Blocks per stage: the 24 complex 11x11 filters, the RBF weights and lambda_t, all
// updated from one gradient evaluation at the inertial point (alpha = beta):
//   x^{k+1} = P(z^k - tau g),   z^{k+1} = x^{k+1} + alpha_{k+1} (x^{k+1} - x^k)
// with P the projection onto the constraints: each filter zero-mean over its taps with
// Euclidean norm <= 1 (projection onto the zero-mean subspace, then onto the unit ball: exact,
// since the ball is centred in the subspace), lambda_t >= 0, RBF weights free.
//
// One CTA per (stage, filter) and one per stage for its RBF weights and lambda; block sums are
// formed in a fixed order (deterministic).
#include "plan.cuh"

namespace {

constexpr int kTaps = VARNET_KSIZE * VARNET_KSIZE;      // 121
constexpr int kFilt = VARNET_NK * 2 * kTaps;           // real-form filters of one stage
constexpr int kStage = kFilt + VARNET_NK * VARNET_NW + 1;
constexpr int kThreads = 256;                           // >= 2 * kTaps: one value per thread

// Fixed-order block sum of one value per thread (kThreads = 8 warps).
__device__ __forceinline__ float block_sum(float v, float* sh) {
  v = warp_sum_f(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
  return t;
}

__global__ void __launch_bounds__(kThreads)
k_ipalm_varnet(float* __restrict__ z, float* __restrict__ g, float* __restrict__ x, float tau_f,
               float tau_r, float tau_l, float alpha) {
  __shared__ float sh[kThreads / 32];
  const int t = blockIdx.y;                   // stage
  float* zs = z + (size_t)t * kStage;
  float* gs = g + (size_t)t * kStage;
  float* xs = x + (size_t)t * kStage;
  if (blockIdx.x < VARNET_NK) {
    // filter i: real form w[i][0][.] = Re k_i, w[i][1][.] = -Im k_i (taps of one channel
    // contiguous); zero mean of k_i is zero mean of both channels, ||k_i|| = ||w[i]||
    const int i = blockIdx.x;
    const int j = threadIdx.x;                // 0..241 valid
    const bool valid = j < 2 * kTaps;
    const int o = i * 2 * kTaps + j;
    float v = 0.f;
    if (valid) v = zs[o] - tau_f * gs[o];
    const bool ch1 = j >= kTaps;
    const float s0 = block_sum(valid && !ch1 ? v : 0.f, sh);
    const float s1 = block_sum(valid && ch1 ? v : 0.f, sh);
    if (valid) v -= (ch1 ? s1 : s0) * (1.f / kTaps);
    const float n2 = block_sum(valid ? v * v : 0.f, sh);
    if (n2 > 1.f) v *= rsqrtf(n2);
    if (valid) {
      const float xo = xs[o];
      xs[o] = v;
      zs[o] = fmaf(alpha, v - xo, v);
      gs[o] = 0.f;
    }
  } else {
    // RBF weights (free) and lambda_t (>= 0)
    for (int j = threadIdx.x; j < VARNET_NK * VARNET_NW + 1; j += kThreads) {
      const int o = kFilt + j;
      const bool lam = j == VARNET_NK * VARNET_NW;
      float v = zs[o] - (lam ? tau_l : tau_r) * gs[o];
      if (lam) v = fmaxf(v, 0.f);
      const float xo = xs[o];
      xs[o] = v;
      zs[o] = fmaf(alpha, v - xo, v);
      gs[o] = 0.f;
    }
  }
}

}  // namespace

extern "C" int ipalm_update_varnet(float* params, float* grad, float* x, int T, float tau_filters,
                                   float tau_rbf, float tau_lambda, float alpha_next, void* stream) {
  if (!params || !grad || !x) return SENSE_EINVAL_PTR;
  if (T <= 0 || !(tau_filters >= 0.f) || !(tau_rbf >= 0.f) || !(tau_lambda >= 0.f) ||
      !(alpha_next >= 0.f) || !(alpha_next < 1.f))
    return SENSE_EINVAL_ARG;
  if (params == grad || params == x || grad == x) return SENSE_EINVAL_PTR;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_mark("unrolled_misc", st, false);
  k_ipalm_varnet<<<dim3(VARNET_NK + 1, T), kThreads, 0, st>>>(params, grad, x, tau_filters, tau_rbf,
                                                              tau_lambda, alpha_next);
  prof_mark("unrolled_misc", st, true);
  prof_count(1);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}
