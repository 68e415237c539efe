// Variational Network stage (Sec. 2.3.1, Eq. 5), forward and reverse mode:
//
//   x_{t+1} = x_t - sum_i K_i^T Phi_i'(K_i x_t) - lambda_t (A^H A x_t - A^H y)
//
// K_i x = Re(k_i * x): N_k = 24 complex 11x11 filters applied to the complex
// image as two real channels, imaginary part discarded; Phi_i' is a weighted
// sum of N_w = 31 Gaussian radial basis functions with centres on [-1, 1] and
// width equal to their spacing.  Per-stage parameters (float32, 6,553 values):
// real-form filters w[i][c][11][11] (w[i][0] = Re k_i, w[i][1] = -Im k_i),
// RBF weights r[i][31], step size lambda_t.
//
// Arithmetic: convolution inputs and filters in BF16, FP32 accumulation, RBF
// in FP32.  The sum over the 31 Gaussians keeps the 13 centres within 6.5
// widths of z (the others are below e^-21 of the largest term).
//   K       warp-level tensor cores (mma.sync m16n8k16) on an im2col tile built
//           per filter row in shared memory (K = 2 channels x 11 taps, padded to 32);
//   K^T     mma.sync straight from a channels-last halo of the 24 (padded 32)
//           activation channels, 121 taps x 32 channels, N = 8 (2 used);
//   dL/dw   mma.sync per image row: A = u^T (ldmatrix.trans of [w][i]), B = the
//           Hankel matrix B[w][dx] = row[w + dx] of each shifted source row;
//   dL/dr   CUDA cores, per-row partials.
// Every gradient is summed per image row and reduced over rows in a fixed order.
#include <cuda_bf16.h>

#include <cmath>
#include <mutex>

#include "plan.cuh"

namespace {

constexpr int NK = 24;          // filters
constexpr int NW = 31;          // radial basis functions
constexpr int KS = 11;          // filter size
constexpr int KH = KS / 2;      // 5
constexpr int NT = KS * KS;     // 121 taps
constexpr int NPAR = NK * 2 * NT + NK * NW + 1;  // 6553
constexpr int OFF_RBF = NK * 2 * NT;             // 5808
constexpr int OFF_LAM = OFF_RBF + NK * NW;       // 6552
constexpr int CU = 32;          // padded activation channels
constexpr int TILE = 128;       // pixels per row tile
constexpr int HW_ = TILE + 2 * KH;  // 138 halo pixels
constexpr int LDI = 40;         // padded row (bf16) of im2col / halo tiles: conflict-free ldmatrix
constexpr float kMu0 = -1.f;
constexpr float kDelta = 2.f / 30.f;  // centre spacing = width sigma

__device__ __forceinline__ float bfv(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ uint32_t smem32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem32(p)));
}
__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem32(p)));
}
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Index of the centre nearest z, clamped so that the +-6 window stays in int range
// (NaN maps to 0; far-out z leave an empty window: every term is below e^-21).
__device__ __forceinline__ int nearest_centre(float z) {
  const float t = fminf(fmaxf((z - kMu0) * (1.f / kDelta), -64.f), 64.f);
  return __float2int_rn(t);
}

// Phi'(z) and Phi''(z) for one channel.
struct Rbf {
  float d1, d2;
};
__device__ __forceinline__ Rbf rbf_eval(float z, const float* r) {
  const float inv_s2 = 1.f / (kDelta * kDelta);
  const int jc = nearest_centre(z);
  const int j0 = max(jc - 6, 0), j1 = min(jc + 6, NW - 1);
  Rbf o{0.f, 0.f};
  for (int j = j0; j <= j1; ++j) {
    const float d = z - (kMu0 + kDelta * j);
    const float e = expf(-0.5f * d * d * inv_s2);
    o.d1 = fmaf(r[j], e, o.d1);
    o.d2 = fmaf(r[j] * e, -d * inv_s2, o.d2);
  }
  return o;
}

// ------------------------------------------------------------------ packing
// Wd[dy][n][k]: K operand per filter row, k = c * 11 + dx (22 of 32 used), n = filter (24 of 32).
// WT[t][c][k]: K^T operand per halo offset t = (ry, rx), k = filter (24 of 32), flipped taps.
__global__ void k_vn_pack(const float* prm, __nv_bfloat16* wd, __nv_bfloat16* wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < KS * CU * LDI) {
    const int dy = i / (CU * LDI), n = (i / LDI) % CU, k = i % LDI;
    float v = 0.f;
    if (n < NK && k < 2 * KS) {
      const int c = k / KS, dx = k % KS;
      v = prm[(n * 2 + c) * NT + dy * KS + dx];
    }
    wd[i] = __float2bfloat16_rn(v);
  }
  const int j = i - KS * CU * LDI;
  if (j >= 0 && j < NT * 2 * CU) {
    const int t = j / (2 * CU), c = (j / CU) % 2, k = j % CU;
    float v = 0.f;
    if (k < NK) v = prm[(k * 2 + c) * NT + (NT - 1 - t)];
    wt[j] = __float2bfloat16_rn(v);
  }
}

// -------------------------------------------------------------- K (2 -> 24)
// mode 0 (forward stage):  u = Phi'(K x)                         -> u [px][32] bf16
// mode 1 (reverse stage):  z = K x, kg = K g;  u = Phi'(z), v = Phi''(z) kg
//                          -> u, v [px][32] bf16, z, kg [px][24] fp32
struct KArgs {
  int B, H, W, mode;
  const float2* x;
  const float2* g;
  const __nv_bfloat16* wd;
  const float* rbf;  // [24][31]
  __nv_bfloat16* u;
  __nv_bfloat16* v;
  float* z;
  float* kg;
};

constexpr int K_SMEM_HALO = 2 * 2 * KS * HW_ * 2;      // [src][c][row][px] bf16
constexpr int K_SMEM_COL = 2 * TILE * LDI * 2;         // im2col per source
constexpr int K_SMEM_W = KS * CU * LDI * 2;
constexpr int K_SMEM = K_SMEM_HALO + K_SMEM_COL + K_SMEM_W + NK * NW * 4;

__global__ void __launch_bounds__(128) k_vn_K(const KArgs a) {
  extern __shared__ __align__(16) uint8_t dsm[];
  __nv_bfloat16* halo = reinterpret_cast<__nv_bfloat16*>(dsm);                       // [2][2][11][138]
  __nv_bfloat16* col = reinterpret_cast<__nv_bfloat16*>(dsm + K_SMEM_HALO);          // [2][128][40]
  __nv_bfloat16* wd = reinterpret_cast<__nv_bfloat16*>(dsm + K_SMEM_HALO + K_SMEM_COL);
  float* s_r = reinterpret_cast<float*>(dsm + K_SMEM_HALO + K_SMEM_COL + K_SMEM_W);
  const int nsrc = a.mode ? 2 : 1;
  const int bh = blockIdx.y, b = bh / a.H, h = bh % a.H, w0 = blockIdx.x * TILE;
  for (int i = threadIdx.x; i < KS * CU * LDI / 8; i += blockDim.x)
    reinterpret_cast<uint4*>(wd)[i] = reinterpret_cast<const uint4*>(a.wd)[i];
  for (int i = threadIdx.x; i < NK * NW; i += blockDim.x) s_r[i] = a.rbf[i];
  for (int s = 0; s < nsrc; ++s) {
    const float2* src = s ? a.g : a.x;
    for (int i = threadIdx.x; i < KS * HW_; i += blockDim.x) {
      const int r = i / HW_, px = i % HW_;
      const int yy = h - KH + r, xx = w0 - KH + px;
      float2 v = make_float2(0.f, 0.f);
      if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) v = src[((size_t)b * a.H + yy) * a.W + xx];
      halo[((s * 2 + 0) * KS + r) * HW_ + px] = __float2bfloat16_rn(v.x);
      halo[((s * 2 + 1) * KS + r) * HW_ + px] = __float2bfloat16_rn(v.y);
    }
  }
  // columns 22..39 of the im2col tiles stay zero
  for (int i = threadIdx.x; i < 2 * TILE * LDI; i += blockDim.x) col[i] = __float2bfloat16_rn(0.f);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tig = lane & 3, mi = lane >> 3, rr = lane & 7;
  float acc[2][2][4][4];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[s][mt][nt][e] = 0.f;

#pragma unroll 1
  for (int dy = 0; dy < KS; ++dy) {
    for (int i = threadIdx.x; i < nsrc * TILE * 2 * KS; i += blockDim.x) {
      const int s = i / (TILE * 2 * KS), rem = i % (TILE * 2 * KS);
      const int m = rem / (2 * KS), k = rem % (2 * KS);
      const int c = k / KS, dx = k % KS;
      col[(s * TILE + m) * LDI + k] = halo[((s * 2 + c) * KS + dy) * HW_ + m + dx];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 32; kk += 16) {
      uint32_t bfr[2][4];
#pragma unroll
      for (int np = 0; np < 2; ++np) {  // n-tile pairs (16 filters)
        const int n = np * 16 + (mi >> 1) * 8 + rr, k = kk + (mi & 1) * 8;
        ldsm4(bfr[np], wd + (dy * CU + n) * LDI + k);
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (s >= nsrc) break;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          uint32_t af[4];
          const int m = warp * 32 + mt * 16 + (mi & 1) * 8 + rr, k = kk + (mi >> 1) * 8;
          ldsm4(af, col + (s * TILE + m) * LDI + k);
#pragma unroll
          for (int np = 0; np < 2; ++np) {
            mma16816(acc[s][mt][2 * np], af, bfr[np][0], bfr[np][1]);
            mma16816(acc[s][mt][2 * np + 1], af, bfr[np][2], bfr[np][3]);
          }
        }
      }
    }
    __syncthreads();
  }
  // epilogue: element (pixel row, filter col) of each fragment
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int w = w0 + warp * 32 + mt * 16 + gid + half * 8;
      if (w >= a.W) continue;
      const size_t p = ((size_t)b * a.H + h) * a.W + w;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int i0 = nt * 8 + 2 * tig;
        float uo[2] = {0.f, 0.f}, vo[2] = {0.f, 0.f};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int i = i0 + e;
          if (i >= NK) continue;
          const float z = acc[0][mt][nt][half * 2 + e];
          const Rbf f = rbf_eval(z, s_r + i * NW);
          uo[e] = f.d1;
          if (a.mode) {
            const float kgv = acc[1][mt][nt][half * 2 + e];
            vo[e] = f.d2 * kgv;
            a.z[p * NK + i] = z;
            a.kg[p * NK + i] = kgv;
          }
        }
        *reinterpret_cast<uint32_t*>(a.u + p * CU + i0) =
            pack2(__float2bfloat16_rn(uo[0]), __float2bfloat16_rn(uo[1]));
        if (a.mode)
          *reinterpret_cast<uint32_t*>(a.v + p * CU + i0) =
              pack2(__float2bfloat16_rn(vo[0]), __float2bfloat16_rn(vo[1]));
      }
    }
}

// ------------------------------------------------------------ K^T (24 -> 2)
// out = base - K^T(src) - lambda (n - c)   (c may be NULL)
struct KTArgs {
  int B, H, W;
  const __nv_bfloat16* src;  // [px][32]
  const __nv_bfloat16* wt;   // [121][2][32]
  const float2* base;
  const float2* n;
  const float2* c;
  const float* lam;
  float2* out;
};

constexpr int KT_SMEM_HALO = KS * HW_ * LDI * 2;
constexpr int KT_SMEM = KT_SMEM_HALO + NT * 2 * CU * 2;

__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem32(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

__global__ void __launch_bounds__(128) k_vn_KT(const KTArgs a) {
  extern __shared__ __align__(16) uint8_t dsm[];
  __nv_bfloat16* halo = reinterpret_cast<__nv_bfloat16*>(dsm);  // [11][138][40]
  __nv_bfloat16* wt = reinterpret_cast<__nv_bfloat16*>(dsm + KT_SMEM_HALO);
  const int bh = blockIdx.y, b = bh / a.H, h = bh % a.H, w0 = blockIdx.x * TILE;
  for (int i = threadIdx.x; i < NT * 2 * CU / 8; i += blockDim.x) cp16(wt + i * 8, a.wt + i * 8, true);
  for (int i = threadIdx.x; i < KS * HW_ * 4; i += blockDim.x) {
    const int q = i & 3, px = (i >> 2) % HW_, r = (i >> 2) / HW_;
    const int yy = h - KH + r, xx = w0 - KH + px;
    const bool ok = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
    cp16(halo + (r * HW_ + px) * LDI + q * 8,
         a.src + (ok ? (((size_t)b * a.H + yy) * a.W + xx) * CU + q * 8 : 0), ok);
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tig = lane & 3, mi = lane >> 3, rr = lane & 7;
  float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll 1
  for (int t = 0; t < NT; ++t) {
    const int ry = t / KS, rx = t % KS;
#pragma unroll
    for (int kk = 0; kk < CU; kk += 16) {
      uint32_t b0 = 0u, b1 = 0u;
      if (gid < 2) {
        b0 = *reinterpret_cast<const uint32_t*>(wt + (t * 2 + gid) * CU + kk + 2 * tig);
        b1 = *reinterpret_cast<const uint32_t*>(wt + (t * 2 + gid) * CU + kk + 8 + 2 * tig);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        uint32_t af[4];
        const int m = warp * 32 + mt * 16 + (mi & 1) * 8 + rr, k = kk + (mi >> 1) * 8;
        ldsm4(af, halo + (ry * HW_ + m + rx) * LDI + k);
        mma16816(d[mt], af, b0, b1);
      }
    }
  }
  if (tig == 0) {
    const float lam = a.lam[0];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int w = w0 + warp * 32 + mt * 16 + gid + half * 8;
        if (w >= a.W) continue;
        const size_t p = ((size_t)b * a.H + h) * a.W + w;
        const float2 bv = a.base[p], nv = a.n[p];
        const float2 cv = a.c ? a.c[p] : make_float2(0.f, 0.f);
        a.out[p] = make_float2(bv.x - d[mt][2 * half] - lam * (nv.x - cv.x),
                               bv.y - d[mt][2 * half + 1] - lam * (nv.y - cv.y));
      }
  }
}

// ------------------------------------------------------- filter gradients
// Per image row h:  G[i][c][dy][dx] = sum_w u[h,w][i] gs[h+dy-5, w+dx-5][c]
//                                    + v[h,w][i] xs[h+dy-5, w+dx-5][c]
// (the filter gradient is -G).  A = u^T, v^T (ldmatrix.trans of [w][32]);
// B[w][dx] = row[w + dx] of a zero-padded BF16 source row.  Warp w takes the
// (c, dy) pairs w, w + 4, ...; each pair is a 32 x 16 (i x dx) tile.
constexpr int WG_MAXW = 512;
constexpr int WG_ROW = WG_MAXW + 2 * KH + 16;  // padded source row
__host__ __device__ constexpr int wg_smem(int W) {
  return 2 * ((W + 15) / 16 * 16) * LDI * 2 + 2 * 2 * KS * WG_ROW * 2;
}

__global__ void __launch_bounds__(128) k_vn_wgrad(int B, int H, int W, const __nv_bfloat16* u,
                                                  const __nv_bfloat16* v, const float2* gs, const float2* xs,
                                                  float* partial) {
  extern __shared__ __align__(16) uint8_t dsm[];
  const int Wp = (W + 15) / 16 * 16;
  __nv_bfloat16* su = reinterpret_cast<__nv_bfloat16*>(dsm);  // [2][Wp][40]: u, v
  __nv_bfloat16* srow = su + 2 * Wp * LDI;                   // [2 src][2 c][11][WG_ROW]
  const int b = blockIdx.x / H, h = blockIdx.x % H;
  for (int i = threadIdx.x; i < 2 * Wp * 4; i += blockDim.x) {
    const int s = i / (Wp * 4), w = (i / 4) % Wp, q = i & 3;
    const __nv_bfloat16* src = s ? v : u;
    cp16(su + (s * Wp + w) * LDI + q * 8, src + (w < W ? (((size_t)b * H + h) * W + w) * CU + q * 8 : 0),
         w < W);
  }
  for (int i = threadIdx.x; i < 2 * KS * WG_ROW; i += blockDim.x) {
    const int s = i / (KS * WG_ROW), r = (i / WG_ROW) % KS, j = i % WG_ROW;
    const int yy = h - KH + r, xx = j - KH;
    const float2* src = s ? xs : gs;
    float2 val = make_float2(0.f, 0.f);
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) val = src[((size_t)b * H + yy) * W + xx];
    srow[((s * 2 + 0) * KS + r) * WG_ROW + j] = __float2bfloat16_rn(val.x);
    srow[((s * 2 + 1) * KS + r) * WG_ROW + j] = __float2bfloat16_rn(val.y);
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tig = lane & 3, mi = lane >> 3, rr = lane & 7;
  float acc[6][2][2][4];
#pragma unroll
  for (int q = 0; q < 6; ++q)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[q][mt][nt][e] = 0.f;
#pragma unroll 1
  for (int w0 = 0; w0 < Wp; w0 += 16) {
    uint32_t af[2][2][4];  // [u|v][m-tile]
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        // A[m = i][k = w] from storage [w][i]: matrices (m0,k0) (m8,k0) (m0,k8) (m8,k8)
        const int m0 = mt * 16 + (mi & 1) * 8, k0 = (mi >> 1) * 8;
        ldsm4t(af[s][mt], su + (s * Wp + w0 + k0 + rr) * LDI + m0);
      }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int pc = warp + 4 * q;  // (c, dy) pair
      if (pc >= 2 * KS) break;
      const int c = pc / KS, dy = pc % KS;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        // the u term pairs with the gradient rows, the v term with the image rows
        const __nv_bfloat16* row = srow + ((s * 2 + c) * KS + dy) * WG_ROW + w0;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int n = nt * 8 + gid;
          const int k = 2 * tig;
          const uint32_t b0 = pack2(row[k + n], row[k + 1 + n]);
          const uint32_t b1 = pack2(row[k + 8 + n], row[k + 9 + n]);
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) mma16816(acc[q][mt][nt], af[s][mt], b0, b1);
        }
      }
    }
  }
  // partial per row: [i][c][dy][dx] (24 x 2 x 11 x 11), D rows = i, cols = dx
  float* out = partial + (size_t)blockIdx.x * (NK * 2 * NT);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int pc = warp + 4 * q;
    if (pc >= 2 * KS) break;
    const int c = pc / KS, dy = pc % KS;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = mt * 16 + gid + (e >= 2 ? 8 : 0);
          const int dx = nt * 8 + 2 * tig + (e & 1);
          if (i < NK && dx < KS) out[(i * 2 + c) * NT + dy * KS + dx] = acc[q][mt][nt][e];
        }
  }
}

// RBF weight gradient partial per row: P[i][j] = sum_w kg[w][i] * phi_j(z[w][i]).
// Thread (i, q): pixels w = q, q + 8, ...; the eight q-partials are added in order.
__global__ void __launch_bounds__(192) k_vn_rbfgrad(int B, int H, int W, const float* z, const float* kg,
                                                    float* partial) {
  __shared__ float s_p[8][NK * NW];
  const int i = threadIdx.x % NK, q = threadIdx.x / NK;  // 24 x 8
  const int b = blockIdx.x / H, h = blockIdx.x % H;
  float acc[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) acc[j] = 0.f;
  const float inv_s2 = 1.f / (kDelta * kDelta);
  for (int w = q; w < W; w += 8) {
    const size_t p = ((size_t)b * H + h) * W + w;
    const float zz = z[p * NK + i], g = kg[p * NK + i];
    const int jc = nearest_centre(zz);
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      if (j < jc - 6 || j > jc + 6) continue;
      const float d = zz - (kMu0 + kDelta * j);
      acc[j] = fmaf(g, expf(-0.5f * d * d * inv_s2), acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < NW; ++j) s_p[q][i * NW + j] = acc[j];
  __syncthreads();
  float* out = partial + (size_t)blockIdx.x * (NK * NW);
  for (int k = threadIdx.x; k < NK * NW; k += blockDim.x) {
    float s = 0.f;
    for (int qq = 0; qq < 8; ++qq) s += s_p[qq][k];
    out[k] = s;
  }
}

// grad[k] += scale * sum over rows (fixed order: eight interleaved row groups, then in order)
__global__ void __launch_bounds__(256) k_vn_reduce(const float* partial, int nrows, int ncols, float scale,
                                                   float* grad) {
  __shared__ float s_part[8][32];
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (col < ncols)
    for (int r = wg; r < nrows; r += 8) s += partial[(size_t)r * ncols + col];
  s_part[wg][lane] = s;
  __syncthreads();
  if (wg == 0 && col < ncols) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += s_part[k][lane];
    grad[col] += scale * t;
  }
}

// grad_lambda_t -= Re<g, n - c> is a row-dot via the CG helper (launch_dot_rows).

size_t up256(size_t n) { return (n + 255) & ~(size_t)255; }

struct VnLayout {
  size_t wd, wt, u, v, z, kg, n1, n2, part, pdot, total;
};
VnLayout vn_layout(int B, int H, int W) {
  VnLayout L;
  const size_t px = (size_t)B * H * W;
  size_t o = 0;
  L.wd = o; o += up256(KS * CU * LDI * 2);
  L.wt = o; o += up256(NT * 2 * CU * 2);
  L.u = o; o += up256(px * CU * 2);
  L.v = o; o += up256(px * CU * 2);
  L.z = o; o += up256(px * NK * 4);
  L.kg = o; o += up256(px * NK * 4);
  L.n1 = o; o += up256(px * 8);
  L.n2 = o; o += up256(px * 8);
  L.part = o; o += up256((size_t)B * H * NK * 2 * NT * 4);
  L.pdot = o; o += 256;
  L.total = o;
  return L;
}

int vn_prepare() {
  static int state = 0;
  static std::mutex mu;
  std::lock_guard<std::mutex> l(mu);
  if (state == 0)
    state = (cudaFuncSetAttribute(k_vn_K, cudaFuncAttributeMaxDynamicSharedMemorySize, K_SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_vn_KT, cudaFuncAttributeMaxDynamicSharedMemorySize, KT_SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_vn_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, wg_smem(WG_MAXW)) ==
                 cudaSuccess)
                ? 1
                : -1;
  return state == 1 ? SENSE_OK : SENSE_ECUDA;
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int vn_check(sense_plan p, const float* prm, const void* AHy, const void* xt, void* ws, size_t ws_bytes) {
  if (!p || !prm || !AHy || !xt || !ws || !al16(AHy) || !al16(xt) || ((uintptr_t)ws & 255u)) return SENSE_EINVAL_PTR;
  if (p->W > WG_MAXW || (long long)p->B * p->H > 65535) return SENSE_EUNSUPPORTED;
  if (ws_bytes < vn_layout(p->B, p->H, p->W).total) return SENSE_EWORKSPACE;
  return vn_prepare();
}

void vn_pack(const float* prm, uint8_t* ws, const VnLayout& L, cudaStream_t st) {
  const int n = KS * CU * LDI + NT * 2 * CU;
  prof_mark("vn_misc", st, false);
  k_vn_pack<<<(n + 255) / 256, 256, 0, st>>>(prm, reinterpret_cast<__nv_bfloat16*>(ws + L.wd),
                                             reinterpret_cast<__nv_bfloat16*>(ws + L.wt));
  prof_mark("vn_misc", st, true);
}

int launch_K(sense_plan p, int mode, const float* prm, const float2* x, const float2* g, uint8_t* ws,
             const VnLayout& L) {
  KArgs a;
  a.B = p->B; a.H = p->H; a.W = p->W; a.mode = mode;
  a.x = x; a.g = g;
  a.wd = reinterpret_cast<const __nv_bfloat16*>(ws + L.wd);
  a.rbf = prm + OFF_RBF;
  a.u = reinterpret_cast<__nv_bfloat16*>(ws + L.u);
  a.v = reinterpret_cast<__nv_bfloat16*>(ws + L.v);
  a.z = reinterpret_cast<float*>(ws + L.z);
  a.kg = reinterpret_cast<float*>(ws + L.kg);
  const char* grp = mode ? "vn_Kbwd" : "vn_K";
  prof_mark(grp, p->stream, false);
  k_vn_K<<<dim3((p->W + TILE - 1) / TILE, p->B * p->H), 128, K_SMEM, p->stream>>>(a);
  prof_mark(grp, p->stream, true);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int launch_KT(sense_plan p, const __nv_bfloat16* src, const float* prm, const float2* base, const float2* n,
              const float2* c, float2* out, uint8_t* ws, const VnLayout& L) {
  KTArgs a;
  a.B = p->B; a.H = p->H; a.W = p->W;
  a.src = src;
  a.wt = reinterpret_cast<const __nv_bfloat16*>(ws + L.wt);
  a.base = base; a.n = n; a.c = c; a.lam = prm + OFF_LAM; a.out = out;
  prof_mark("vn_KT", p->stream, false);
  k_vn_KT<<<dim3((p->W + TILE - 1) / TILE, p->B * p->H), 128, KT_SMEM, p->stream>>>(a);
  prof_mark("vn_KT", p->stream, true);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

// Normal operator without lambda (A^H A x) through the plan's own path.
int normal0(sense_plan p, const float2* x, float2* out) { return sense_normal(p, x, out, 0.f); }

// d/dlambda of the stage: -Re<g, n - c>, added to grad[OFF_LAM] (float32).
__global__ void k_vn_addlam(const double* d, float* g) { g[OFF_LAM] += (float)(-d[0]); }

}  // namespace

extern "C" {

size_t varnet_workspace_bytes(int B, int H, int W) {
  if (B <= 0 || H <= 0 || W <= 0) return 0;
  return vn_layout(B, H, W).total;
}

int varnet_param_count(void) { return NPAR; }

int varnet_stage(sense_plan p, const float* prm, const void* AHy, const void* x_t, void* x_next, void* ws,
                 size_t ws_bytes) {
  if (int e = vn_check(p, prm, AHy, x_t, ws, ws_bytes)) return e;
  if (!x_next || !al16(x_next) || x_next == x_t) return SENSE_EINVAL_PTR;
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  const VnLayout L = vn_layout(p->B, p->H, p->W);
  const float2* x = static_cast<const float2*>(x_t);
  float2* n1 = reinterpret_cast<float2*>(w8 + L.n1);
  vn_pack(prm, w8, L, p->stream);
  if (int e = normal0(p, x, n1)) return e;
  if (int e = launch_K(p, 0, prm, x, nullptr, w8, L)) return e;
  if (int e = launch_KT(p, reinterpret_cast<const __nv_bfloat16*>(w8 + L.u), prm, x, n1,
                        static_cast<const float2*>(AHy), static_cast<float2*>(x_next), w8, L))
    return e;
  prof_count(3);
  return SENSE_OK;
}

int varnet_stage_backward(sense_plan p, const float* prm, const void* AHy, const void* x_t,
                          const void* grad_next, void* grad_t, float* grad_prm, void* ws, size_t ws_bytes) {
  if (int e = vn_check(p, prm, AHy, x_t, ws, ws_bytes)) return e;
  if (!grad_next || !grad_t || !grad_prm || !al16(grad_next) || !al16(grad_t) || grad_t == grad_next)
    return SENSE_EINVAL_PTR;
  if (!p->ws) return SENSE_EWORKSPACE;  // the lambda-gradient dot uses the plan's workspace
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  const VnLayout L = vn_layout(p->B, p->H, p->W);
  const float2* x = static_cast<const float2*>(x_t);
  const float2* g = static_cast<const float2*>(grad_next);
  float2* n1 = reinterpret_cast<float2*>(w8 + L.n1);
  float2* n2 = reinterpret_cast<float2*>(w8 + L.n2);
  double* pdot = reinterpret_cast<double*>(w8 + L.pdot);
  float* part = reinterpret_cast<float*>(w8 + L.part);
  const int rows = p->B * p->H;
  vn_pack(prm, w8, L, p->stream);
  // grad lambda_t = -Re<g, A^H A x - A^H y>
  if (int e = normal0(p, x, n1)) return e;
  if (int e = launch_dot_rows(p, g, n1, static_cast<const float2*>(AHy), pdot, 1, 0)) return e;
  prof_mark("vn_misc", p->stream, false);
  k_vn_addlam<<<1, 1, 0, p->stream>>>(pdot, grad_prm);
  prof_mark("vn_misc", p->stream, true);
  // z = K x, kg = K g, u = Phi'(z), v = Phi''(z) kg
  if (int e = launch_K(p, 1, prm, x, g, w8, L)) return e;
  // filter gradient: -(sum u (x) g_shift + v (x) x_shift); reads g and x before grad_t is written
  prof_mark("vn_wgrad", p->stream, false);
  k_vn_wgrad<<<rows, 128, wg_smem(p->W), p->stream>>>(
      p->B, p->H, p->W, reinterpret_cast<const __nv_bfloat16*>(w8 + L.u),
      reinterpret_cast<const __nv_bfloat16*>(w8 + L.v), g, x, part);
  k_vn_reduce<<<(NK * 2 * NT + 31) / 32, 256, 0, p->stream>>>(part, rows, NK * 2 * NT, -1.f, grad_prm);
  prof_mark("vn_wgrad", p->stream, true);
  // RBF weight gradient: -sum kg phi_j(z)
  prof_mark("vn_rbfgrad", p->stream, false);
  k_vn_rbfgrad<<<rows, 192, 0, p->stream>>>(p->B, p->H, p->W, reinterpret_cast<const float*>(w8 + L.z),
                                            reinterpret_cast<const float*>(w8 + L.kg), part);
  k_vn_reduce<<<(NK * NW + 31) / 32, 256, 0, p->stream>>>(part, rows, NK * NW, -1.f, grad_prm + OFF_RBF);
  prof_mark("vn_rbfgrad", p->stream, true);
  // grad_t = g - K^T v - lambda A^H A g
  if (int e = normal0(p, g, n2)) return e;
  if (int e = launch_KT(p, reinterpret_cast<const __nv_bfloat16*>(w8 + L.v), prm, g, n2, nullptr,
                        static_cast<float2*>(grad_t), w8, L))
    return e;
  prof_count(8);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

}  // extern "C"
