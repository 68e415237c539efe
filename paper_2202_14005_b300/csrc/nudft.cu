// Non-uniform DFT pair of non-Cartesian SENSE by direct summation (Sec. 2.3.3: A^H y of the
// measured non-Cartesian samples initialises the networks; the forward simulates such samples):
//   forward  y[b][c][m] = (H W)^{-1/2} sum_n S_c(n) x(n) exp(-2 pi i (ky_m n'_y / H + kx_m n'_x / W))
//   adjoint  x[b][n]    = (H W)^{-1/2} sum_c conj(S_c(n)) sum_m y[b][c][m] exp(+2 pi i (...))
// with centred image coordinates n' = n - (H/2, W/2) and k in grid units, so on-grid samples
// give the centred unitary DFT of the Cartesian operator.  Cost O(M H W C) per slice: these are
// set-up calls (one per scan), like the PSF.
//
// Phasors: exp(2 pi i k n / L) for a float k and an integer n is reduced exactly in FP32 before
// the sine and cosine: k n = hi + lo exactly (fma), hi - q L is exact for the integer
// q = rint(hi / L), so the phase in turns, (hi - q L + lo) / L in [-1/2, 1/2], carries one
// rounding.  The 2-D phasor of a (sample, pixel) pair is the product of its row and column
// phasors.  Sums: FP32 over blocks of 256 terms, then FP64.
#include "plan.cuh"

namespace {

constexpr int kTR = 8, kTC = 32;   // pixel tile: 8 rows x 32 columns (one pixel per thread)
constexpr int kChunk = 32;         // samples staged per step
constexpr int kCG = 6;             // coils per pass (12 and 15 coils: whole passes)

__device__ __forceinline__ float2 phasor(float k, int n, int L, float sign) {
  const float fn = (float)n;
  const float hi = k * fn;
  const float lo = fmaf(k, fn, -hi);
  const float q = rintf(hi / (float)L);
  const float r = fmaf(-q, (float)L, hi) + lo;
  float s, c;
  sincospif(2.f * (r / (float)L), &s, &c);
  return make_float2(c, sign * s);
}

// Adjoint: one CTA per 8 x 32 pixel tile of one slice, one pixel per thread.  Per chunk of 32
// samples the CTA stages the row phasors of its 8 rows, the column phasors of its 32 columns and
// the samples of the pass's coils.
__global__ void __launch_bounds__(256) k_nudft_adjoint(int M, int C, int H, int W, const float* __restrict__ traj,
                                                     const float2* __restrict__ maps,
                                                     const float2* __restrict__ y, float2* __restrict__ x) {
  __shared__ float2 ey[kChunk][kTR], ex[kChunk][kTC], ys[kCG][kChunk];
  const int tc = threadIdx.x & (kTC - 1), tr = threadIdx.x / kTC;
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * kTR, c0 = blockIdx.x * kTC;
  const int row = r0 + tr, col = c0 + tc;
  const bool inside = row < H && col < W;
  const float scale = rsqrtf((float)H * (float)W);
  float2 out = make_float2(0.f, 0.f);
  for (int cb = 0; cb < C; cb += kCG) {
    const int nc = min(kCG, C - cb);
    double ar[kCG], ai[kCG];
    float fr[kCG], fi[kCG];
#pragma unroll
    for (int k = 0; k < kCG; ++k) { ar[k] = ai[k] = 0.0; fr[k] = fi[k] = 0.f; }
    for (int m0 = 0; m0 < M; m0 += kChunk) {
      __syncthreads();
      for (int i = threadIdx.x; i < kChunk * (kTR + kTC); i += blockDim.x) {
        const int mm = i / (kTR + kTC), j = i - mm * (kTR + kTC), m = m0 + mm;
        float2 v = make_float2(0.f, 0.f);
        if (m < M) {
          if (j < kTR) v = phasor(traj[2 * m], r0 + j - H / 2, H, 1.f);
          else v = phasor(traj[2 * m + 1], c0 + (j - kTR) - W / 2, W, 1.f);
        }
        if (j < kTR) ey[mm][j] = v;
        else ex[mm][j - kTR] = v;
      }
      for (int i = threadIdx.x; i < kCG * kChunk; i += blockDim.x) {
        const int k = i / kChunk, mm = i - k * kChunk, m = m0 + mm;
        ys[k][mm] = (k < nc && m < M) ? y[((size_t)b * C + cb + k) * M + m] : make_float2(0.f, 0.f);
      }
      __syncthreads();
#pragma unroll 4
      for (int mm = 0; mm < kChunk; ++mm) {
        const float2 p = cmul(ey[mm][tr], ex[mm][tc]);
#pragma unroll
        for (int k = 0; k < kCG; ++k) {
          const float2 v = ys[k][mm];
          fr[k] = fmaf(v.x, p.x, fmaf(-v.y, p.y, fr[k]));
          fi[k] = fmaf(v.x, p.y, fmaf(v.y, p.x, fi[k]));
        }
      }
      if (((m0 / kChunk) & 7) == 7 || m0 + kChunk >= M) {  // fold every 256 samples into FP64
#pragma unroll
        for (int k = 0; k < kCG; ++k) {
          ar[k] += fr[k];
          ai[k] += fi[k];
          fr[k] = fi[k] = 0.f;
        }
      }
    }
    if (inside) {
#pragma unroll
      for (int k = 0; k < kCG; ++k) {
        if (k < nc) {
          const float2 s = maps[(((size_t)b * C + cb + k) * H + row) * W + col];
          const float2 u = make_float2((float)ar[k], (float)ai[k]);
          out = cfmac(s, u, out);  // conj(S_c) u_c
        }
      }
    }
  }
  if (inside) x[((size_t)b * H + row) * W + col] = make_float2(out.x * scale, out.y * scale);
}

// Forward: one CTA per 256 samples of one slice, one sample per thread.  Per 8 x 32 pixel tile
// the CTA stages u_c = S_c x for the pass's coils; each thread forms its sample's 8 row phasors
// once per tile and one column phasor per column.
__global__ void __launch_bounds__(256) k_nudft_forward(int M, int C, int H, int W, const float* __restrict__ traj,
                                                     const float2* __restrict__ maps,
                                                     const float2* __restrict__ x, float2* __restrict__ y) {
  __shared__ float2 us[kCG][kTR * kTC];
  const int b = blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = m < M;
  const float ky = valid ? traj[2 * m] : 0.f, kx = valid ? traj[2 * m + 1] : 0.f;
  const float scale = rsqrtf((float)H * (float)W);
  for (int cb = 0; cb < C; cb += kCG) {
    const int nc = min(kCG, C - cb);
    double ar[kCG], ai[kCG];
#pragma unroll
    for (int k = 0; k < kCG; ++k) ar[k] = ai[k] = 0.0;
    for (int r0 = 0; r0 < H; r0 += kTR) {
      float2 ey[kTR];
#pragma unroll
      for (int r = 0; r < kTR; ++r) ey[r] = phasor(ky, r0 + r - H / 2, H, -1.f);
      for (int c0 = 0; c0 < W; c0 += kTC) {
        __syncthreads();
        {
          const int tr = threadIdx.x / kTC, tc = threadIdx.x & (kTC - 1);
          const int row = r0 + tr, col = c0 + tc;
          const bool inside = row < H && col < W;
          const float2 xv = inside ? x[((size_t)b * H + row) * W + col] : make_float2(0.f, 0.f);
#pragma unroll
          for (int k = 0; k < kCG; ++k) {
            float2 u = make_float2(0.f, 0.f);
            if (inside && k < nc) u = cmul(maps[(((size_t)b * C + cb + k) * H + row) * W + col], xv);
            us[k][threadIdx.x] = u;
          }
        }
        __syncthreads();
        float fr[kCG], fi[kCG];
#pragma unroll
        for (int k = 0; k < kCG; ++k) fr[k] = fi[k] = 0.f;
        for (int tc = 0; tc < kTC; ++tc) {
          const float2 exv = phasor(kx, c0 + tc - W / 2, W, -1.f);
#pragma unroll
          for (int r = 0; r < kTR; ++r) {
            const float2 p = cmul(ey[r], exv);
#pragma unroll
            for (int k = 0; k < kCG; ++k) {
              const float2 u = us[k][r * kTC + tc];
              fr[k] = fmaf(u.x, p.x, fmaf(-u.y, p.y, fr[k]));
              fi[k] = fmaf(u.x, p.y, fmaf(u.y, p.x, fi[k]));
            }
          }
        }
#pragma unroll
        for (int k = 0; k < kCG; ++k) {
          ar[k] += fr[k];
          ai[k] += fi[k];
        }
      }
    }
    if (valid) {
#pragma unroll
      for (int k = 0; k < kCG; ++k)
        if (k < nc)
          y[((size_t)b * C + cb + k) * M + m] = make_float2((float)ar[k] * scale, (float)ai[k] * scale);
    }
  }
}

int check_args(const float* traj, int M, int B, int C, int H, int W, const void* maps, const void* a,
               const void* o) {
  if (M <= 0 || B <= 0 || C <= 0 || H <= 0 || W <= 0 || (H & 1) || (W & 1)) return SENSE_EINVAL_SHAPE;
  if (!traj || !maps || !a || !o || ((uintptr_t)traj & 7u) || ((uintptr_t)maps & 7u) ||
      ((uintptr_t)a & 7u) || ((uintptr_t)o & 7u) || a == o)
    return SENSE_EINVAL_PTR;
  if (H > 4096 || W > 4096 || (long long)B * C * M > (1ll << 40)) return SENSE_EUNSUPPORTED;
  return SENSE_OK;
}

}  // namespace

extern "C" int sense_nudft_forward(const float* traj, int M, int B, int C, int H, int W, const void* maps,
                                   const void* x, void* y, void* stream) {
  if (int e = check_args(traj, M, B, C, H, W, maps, x, y)) return e;
  const dim3 g((M + 255) / 256, B);
  k_nudft_forward<<<g, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      M, C, H, W, traj, static_cast<const float2*>(maps), static_cast<const float2*>(x), static_cast<float2*>(y));
  prof_count(1);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

extern "C" int sense_nudft_adjoint(const float* traj, int M, int B, int C, int H, int W, const void* maps,
                                   const void* y, void* x, void* stream) {
  if (int e = check_args(traj, M, B, C, H, W, maps, y, x)) return e;
  const dim3 g((W + kTC - 1) / kTC, (H + kTR - 1) / kTR, B);
  k_nudft_adjoint<<<g, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      M, C, H, W, traj, static_cast<const float2*>(maps), static_cast<const float2*>(y), static_cast<float2*>(x));
  prof_count(1);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}
