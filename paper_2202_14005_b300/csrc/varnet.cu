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
// Arithmetic: filters in BF16 (rounded from the float32 parameters at use),
// warp-level tensor cores (mma.sync m16n8k16, FP32 accumulation):
//   K       the image operand is split into three BF16 terms (x = x1 + x2 + x3,
//           the full 24-bit significand), so K x is as accurate as FP32
//           accumulation: the zero-mean filters cancel on smooth images (one
//           BF16 rounding of x costs ~1e-2 relative in K x, two terms ~1e-4,
//           and the RBF tails amplify errors of z by up to (z - mu)/sigma^2).
//           The im2col tile of each source row is built once and serves the
//           output rows it touches (A = pixels x [x1 | x2 | x3 taps], B = filters);
//   Phi'    FP32 over the 13 centres nearest z (the rest are below e^-21 of
//           the largest term), fused into the K epilogue;
//   K^T     from BF16 Phi'(z) (channels-last, 24 of 32 channels): per source
//           row and tap column dx, A = pixels x channels and B = filters x
//           (output row, output channel) for a band of 8 output rows, so one
//           MMA serves 8 rows x 2 channels; the stage combine is its epilogue;
//   dL/dw   mma.sync per image row: A = u^T (ldmatrix.trans of [w][i]), B = the
//           Hankel matrix B[w][dx] = row[w + dx] of each shifted source row;
//   dL/dr   CUDA cores, thread-private shared-memory accumulators per row.
// Every gradient is summed per image row or CTA and reduced in a fixed order.
#include <cuda_bf16.h>

#include <cmath>
#include <mutex>

#include "plan.cuh"
#include "tc.cuh"

namespace {

constexpr int NK = 24;          // filters
constexpr int NW = 31;          // radial basis functions
constexpr int KS = 11;          // filter size
constexpr int KH = KS / 2;      // 5
constexpr int NT = KS * KS;     // 121 taps
constexpr int NPAR = NK * 2 * NT + NK * NW + 1;  // 6553
constexpr int OFF_RBF = NK * 2 * NT;             // 5808
constexpr int OFF_LAM = OFF_RBF + NK * NW;       // 6552
constexpr int CU = 32;          // padded channels of the stored activations u, v
constexpr int TILE = 128;       // pixels per row tile
constexpr int HW_ = TILE + 2 * KH;  // 138 halo pixels
constexpr int LDI = 40;         // padded row (bf16) of channel tiles: conflict-free ldmatrix
constexpr float kMu0 = -1.f;
constexpr float kDelta = 2.f / 30.f;  // centre spacing = width sigma
constexpr float kEinv = 0.36787944117144233f;  // e^-1

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t smem32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem32(p)));
}
__device__ __forceinline__ void ldsm2(uint32_t (&r)[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
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
__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem32(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Phi'(z) = sum_j r_j phi_j(z) and Phi''(z) = -sum_j r_j phi_j(z) (z - mu_j) / sigma^2 with
// phi_j(z) = exp(-(z - mu_j)^2 / (2 sigma^2)), over the 13 centres j0 .. j0 + 12, j0 = jc - 6, around
// the centre jc nearest z; every centre left out is more than 6.5 widths from z, below e^-21 of the
// largest term.  Centres outside 0 .. 30 carry weight zero (the weight rows are padded by RBF_PAD
// on both sides), so the window never shifts and its first term exp(-d_j0^2 / 2), d_j0 in
// [5.5, 6.5], stays a normal float.  With sigma equal to the spacing and d_j = (z - mu_j) / sigma:
// d_{j+1} = d_j - 1 and phi_{j+1} = phi_j exp(d_j - 1/2), so two exponentials start the window and
// products continue it.  Then Phi' = S0 = sum_k t_k and Phi'' = (S1 - (d_j0 - 6) S0) / sigma with
// t_k = r_{j0+k} phi_{j0+k} and S1 = sum_k (k - 6) t_k (|d_j0 - 6| <= 1/2: no cancellation between
// the two parts).  jc is clamped to -6 .. 36 (z beyond: every term below e^-18 r).  The two filters
// of a pair run side by side in packed FP32x2 arithmetic.
constexpr int RBF_WIN = 13;
constexpr int RBF_PAD = 12;                  // zero weights below centre 0 and above centre 30
constexpr int RBF_LD = NW + 2 * RBF_PAD;     // 55: padded weight row
__device__ __forceinline__ int window_start(float z, float& d) {
  const float zc = fminf(fmaxf(z, kMu0 - 8.f * kDelta), -kMu0 + 8.f * kDelta);
  const int jc = min(max(__float2int_rn((zc - kMu0) * (1.f / kDelta)), -6), NW - 1 + 6);
  const int j0 = jc - 6;
  d = (zc - (kMu0 + kDelta * (float)j0)) * (1.f / kDelta);
  return j0;  // -12 .. 30
}

struct Rbf2 {
  float2 d1, d2;
};
// Filters a and b (padded RBF weight rows ra, rb: centre j at ra[j + RBF_PAD]) at z.x and z.y.
__device__ __forceinline__ Rbf2 rbf_eval2(float2 z, const float* ra, const float* rb) {
  float2 d;
  const int ja = window_start(z.x, d.x), jb = window_start(z.y, d.y);
  ra += ja + RBF_PAD;
  rb += jb + RBF_PAD;
  float2 phi = make_float2(expf(-0.5f * d.x * d.x), expf(-0.5f * d.y * d.y));
  float2 rho = make_float2(expf(d.x - 0.5f), expf(d.y - 0.5f));
  const float2 q = make_float2(kEinv, kEinv);
  float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < RBF_WIN; ++k) {
    const float2 t = __fmul2_rn(make_float2(ra[k], rb[k]), phi);
    s0 = __fadd2_rn(s0, t);
    s1 = __ffma2_rn(make_float2((float)(k - 6), (float)(k - 6)), t, s1);
    phi = __fmul2_rn(phi, rho);
    rho = __fmul2_rn(rho, q);
  }
  Rbf2 o;
  o.d1 = s0;
  o.d2 = make_float2((s1.x - (d.x - 6.f) * s0.x) * (1.f / kDelta), (s1.y - (d.y - 6.f) * s0.y) * (1.f / kDelta));
  if (z.x != z.x) o.d1.x = o.d2.x = z.x;  // NaN propagates
  if (z.y != z.y) o.d1.y = o.d2.y = z.y;
  return o;
}

// ------------------------------------------------------------------ packing
constexpr int K_RMAX = 8;       // output rows per K CTA: 8 (one source), 4 (two sources)
constexpr int K_PARTS = 3;      // BF16 terms of the image operand: x = x1 + x2 + x3 (24 bits)
constexpr int K_KP = 24 * K_PARTS;  // im2col columns: per part c0 dx 0..10, c1 dx 0..10, 0, 0
constexpr int K_KSTEPS = (K_KP + 15) / 16;  // 5 MMA k-steps (columns 72..79 zero)
constexpr int K_LD = 88;        // row pitch (bf16) of the im2col tile and the K table (conflict-free)
constexpr int K_W_ELEMS = KS * NK * K_LD;
constexpr int KT_LDW = 40;      // row pitch (bf16) of the K^T table: conflict-free across filter rows
constexpr int KT_W_ELEMS = NT * 2 * KT_LDW;

// wk[dy][n][k]: K operand per filter row, the BF16 filter tap w[n][c][dy][dx] at k = part * 24 +
//   c * 11 + dx for every part; zero elsewhere.
// wn[dy][dx][c][i]: K^T operand, the same taps with the filter index i contiguous (zero for i >= 24;
//   pitch KT_LDW).
__global__ void k_vn_pack(const float* prm, bf16* wk, bf16* wn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < K_W_ELEMS) {
    const int dy = i / (NK * K_LD), n = (i / K_LD) % NK, k = i % K_LD;
    float v = 0.f;
    if (k < K_KP && (k % 24) < 2 * KS) {
      const int kk = k % 24, c = kk / KS, dx = kk % KS;
      v = prm[(n * 2 + c) * NT + dy * KS + dx];
    }
    wk[i] = __float2bfloat16_rn(v);
  }
  const int j = i - K_W_ELEMS;
  if (j >= 0 && j < KT_W_ELEMS) {
    const int t = j / (2 * KT_LDW), c = (j / KT_LDW) % 2, k = j % KT_LDW;
    wn[j] = __float2bfloat16_rn(k < NK ? prm[(k * 2 + c) * NT + t] : 0.f);
  }
}

// -------------------------------------------------------------- K (2 -> 24)
// NSRC = 1 (forward stage):  z = K x, u = Phi'(z)                   -> u [px][32] bf16, z [px][24] fp32
// NSRC = 2 (reverse stage):  z = K x, kg = K g;  u = Phi'(z), v = Phi''(z) kg
//                            -> u, v [px][32] bf16, z, kg [px][24] fp32
// NSRC = 1, ZIN (reverse stage after a forward that kept z and u): the source is g; kg = K g,
//                            v = Phi''(z) kg with z read back -> v, kg
// CTA: 128 pixels x R rows (R = 8 / NSRC), 8 warps x 16 pixels.  Source rows stream through a double-
// buffered FP32 stage (cp.async) into one im2col tile per source; each source row s feeds every
// output row h of the CTA with 0 <= s - h + 5 <= 10 (filter row dy = s - h + 5).  The image
// operand enters as three BF16 terms x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2), so
// K x carries the 24-bit significand of x into the FP32 accumulation.
struct KArgs {
  int B, H, W;
  const float2* x;
  const float2* g;
  const bf16* wk;
  const float* rbf;  // [24][31]
  bf16* u;
  bf16* v;
  float* z;
  float* kg;
};

constexpr int K_THREADS = 256;
constexpr int K_STG = 140;  // staged source row (float2): columns w0 - 6 .. w0 + 133
constexpr int K_PR_LD = 144;  // BF16 part row: the K_STG columns of one part and channel

template <int NSRC>
struct KSmem {
  static constexpr int W_BYTES = K_W_ELEMS * 2;
  static constexpr int COL_BYTES = TILE * K_LD * 2;  // one im2col tile
  static constexpr int STG_BYTES = K_STG * 8;
  static constexpr int OFF_COL = W_BYTES;
  static constexpr int OFF_STG = OFF_COL + NSRC * COL_BYTES;
  static constexpr int PR_BYTES = K_PARTS * 2 * K_PR_LD * 2;  // BF16 part rows of one source row
  static constexpr int OFF_PR = OFF_STG + 2 * NSRC * STG_BYTES;
  static constexpr int OFF_R = OFF_PR + NSRC * PR_BYTES;
  static constexpr int TOTAL = OFF_R + NK * RBF_LD * 4;
};

template <int NSRC, bool ZIN = false>
__global__ void __launch_bounds__(K_THREADS, 2) k_vn_K(const KArgs a) {
  static_assert(!ZIN || NSRC == 1, "z is read back only by the one-source reverse kernel");
  using S = KSmem<NSRC>;
  constexpr int K_R = K_RMAX / NSRC;
  extern __shared__ __align__(16) uint8_t dsm[];
  const bf16* wk = reinterpret_cast<const bf16*>(dsm);
  float* s_r = reinterpret_cast<float*>(dsm + S::OFF_R);
  const int w0 = blockIdx.x * TILE, h0 = blockIdx.y * K_R, b = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gid = lane >> 2, tig = lane & 3, mi = lane >> 3, rr = lane & 7;

  for (int i = tid; i < S::W_BYTES / 16; i += K_THREADS)
    cp16(dsm + i * 16, reinterpret_cast<const uint8_t*>(a.wk) + i * 16, true);
  for (int i = tid; i < NK * RBF_LD; i += K_THREADS) {
    const int j = i % RBF_LD - RBF_PAD;
    s_r[i] = (unsigned)j < (unsigned)NW ? a.rbf[(i / RBF_LD) * NW + j] : 0.f;
  }
  const int s_lo = max(h0 - KH, 0), s_hi = min(h0 + K_R - 1 + KH, a.H - 1);
  const int nrows = s_hi - s_lo + 1;
  auto stage = [&](int k) {
    const int s = s_lo + k, buf = k & 1;
    for (int i = tid; i < NSRC * (K_STG / 2); i += K_THREADS) {
      const int src = i / (K_STG / 2), q = i % (K_STG / 2);
      const int col = w0 - 6 + 2 * q;  // even; W is even, so col + 1 < W whenever col < W
      const bool ok = col >= 0 && col < a.W;
      const float2* base = src ? a.g : a.x;
      cp16(dsm + S::OFF_STG + (buf * NSRC + src) * S::STG_BYTES + q * 16,
           base + (ok ? ((size_t)b * a.H + s) * a.W + col : 0), ok);
    }
  };
  stage(0);
  cp_commit();
  // im2col columns K_KP .. K_LD - 1 are read by the last k-step (against zero taps) but never built
  for (int i = tid; i < NSRC * TILE; i += K_THREADS)
    reinterpret_cast<uint4*>(dsm + S::OFF_COL + (size_t)i * K_LD * 2 + K_KP * 2)[0] = make_uint4(0u, 0u, 0u, 0u);

  float acc[NSRC][K_R][3][4];
#pragma unroll
  for (int s = 0; s < NSRC; ++s)
#pragma unroll
    for (int r = 0; r < K_R; ++r)
#pragma unroll
      for (int nt = 0; nt < 3; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[s][r][nt][e] = 0.f;

#pragma unroll 1
  for (int k = 0; k < nrows; ++k) {
    if (k + 1 < nrows) stage(k + 1);
    cp_commit();
    cp_wait<1>();  // everything but the newest group: source row k and the tables have landed
    __syncthreads();
    // BF16 terms of source row k, once per column: part rows pr[src][part][c][column]
    for (int it = tid; it < NSRC * K_STG; it += K_THREADS) {
      const int src = it / K_STG, j = it % K_STG;
      float2 v = reinterpret_cast<const float2*>(dsm + S::OFF_STG + ((k & 1) * NSRC + src) * S::STG_BYTES)[j];
      bf16* pr = reinterpret_cast<bf16*>(dsm + S::OFF_PR + src * S::PR_BYTES);
#pragma unroll
      for (int part = 0; part < K_PARTS; ++part) {  // x1 = bf16(x), x2 = bf16(x - x1), ... (exact residuals)
        const bf16 re = __float2bfloat16_rn(v.x), im = __float2bfloat16_rn(v.y);
        pr[(part * 2) * K_PR_LD + j] = re;
        pr[(part * 2 + 1) * K_PR_LD + j] = im;
        v.x -= __bfloat162float(re);
        v.y -= __bfloat162float(im);
      }
    }
    __syncthreads();
    // im2col of source row k: item (src, part, pixel m) = taps dx 0..10 of both channels, part-row
    // columns m + 1 .. m + 11 (stage column of tap dx: m + dx + 1).  Consecutive lanes take
    // consecutive pixels of one part (row pitch 176 B: eight lanes store to eight bank groups).
    for (int it = tid; it < NSRC * K_PARTS * TILE; it += K_THREADS) {
      const int src = it / (K_PARTS * TILE), part = (it / TILE) % K_PARTS, m = it % TILE;
      const uint32_t* r0 =
          reinterpret_cast<const uint32_t*>(dsm + S::OFF_PR + src * S::PR_BYTES + (part * 2) * K_PR_LD * 2);
      const uint32_t* r1 = r0 + K_PR_LD / 2;
      const int e0 = m + 1, w0i = e0 >> 1;
      const bool odd = e0 & 1;
      uint32_t A[6], Bw[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        A[q] = r0[w0i + q];
        Bw[q] = r1[w0i + q];
      }
      // align: pair q holds columns e0 + 2q, e0 + 2q + 1 (low half first); element 10 in the low half of [5]
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        A[q] = odd ? __byte_perm(A[q], A[q + 1], 0x5432) : A[q];
        Bw[q] = odd ? __byte_perm(Bw[q], Bw[q + 1], 0x5432) : Bw[q];
      }
      A[5] = odd ? (A[5] >> 16) : (A[5] & 0xffffu);
      Bw[5] = odd ? (Bw[5] >> 16) : (Bw[5] & 0xffffu);
      // row: [c0 taps 0..10 | c1 taps 0..10 | 0 0]
      uint4* dst = reinterpret_cast<uint4*>(dsm + S::OFF_COL + src * S::COL_BYTES + m * K_LD * 2 + part * 48);
      dst[0] = make_uint4(A[0], A[1], A[2], A[3]);
      dst[1] = make_uint4(A[4], A[5] | (Bw[0] << 16), __byte_perm(Bw[0], Bw[1], 0x5432),
                          __byte_perm(Bw[1], Bw[2], 0x5432));
      dst[2] = make_uint4(__byte_perm(Bw[2], Bw[3], 0x5432), __byte_perm(Bw[3], Bw[4], 0x5432),
                          __byte_perm(Bw[4], Bw[5], 0x5432), 0u);
    }
    __syncthreads();
    const int s = s_lo + k;
    const bf16* colb = reinterpret_cast<const bf16*>(dsm + S::OFF_COL);
#pragma unroll 1
    for (int ks = 0; ks < K_KSTEPS; ++ks) {
      uint32_t af[NSRC][4];
#pragma unroll
      for (int src = 0; src < NSRC; ++src)
        ldsm4(af[src], colb + (src * TILE + warp * 16 + (mi & 1) * 8 + rr) * K_LD + ks * 16 + (mi >> 1) * 8);
#pragma unroll
      for (int r = 0; r < K_R; ++r) {
        const int dy = s - (h0 + r) + KH;
        if (dy < 0 || dy >= KS) continue;
        const bf16* wrow = wk + dy * NK * K_LD;
        uint32_t b4[4], b2[2];
        ldsm4(b4, wrow + ((mi >> 1) * 8 + rr) * K_LD + ks * 16 + (mi & 1) * 8);
        ldsm2(b2, wrow + (16 + rr) * K_LD + ks * 16 + (mi & 1) * 8);
#pragma unroll
        for (int src = 0; src < NSRC; ++src) {
          mma16816(acc[src][r][0], af[src], b4[0], b4[1]);
          mma16816(acc[src][r][1], af[src], b4[2], b4[3]);
          mma16816(acc[src][r][2], af[src], b2[0], b2[1]);
        }
      }
    }
  }
  // epilogue: fragment element (pixel gid / gid + 8, filter nt * 8 + 2 tig + e)
#pragma unroll
  for (int r = 0; r < K_R; ++r) {
    const int h = h0 + r;
    if (h >= a.H) continue;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int w = w0 + warp * 16 + gid + half * 8;
      if (w >= a.W) continue;
      const size_t p = ((size_t)b * a.H + h) * a.W + w;
#pragma unroll
      for (int nt = 0; nt < 3; ++nt) {
        const int i0 = nt * 8 + 2 * tig;
        const float2 a0 = make_float2(acc[0][r][nt][half * 2], acc[0][r][nt][half * 2 + 1]);
        if constexpr (ZIN) {  // a0 = K g; z from the forward stage
          const float2 z = *reinterpret_cast<const float2*>(a.z + p * NK + i0);
          const Rbf2 f = rbf_eval2(z, s_r + i0 * RBF_LD, s_r + (i0 + 1) * RBF_LD);
          *reinterpret_cast<uint32_t*>(a.v + p * CU + i0) =
              pack2(__float2bfloat16_rn(f.d2.x * a0.x), __float2bfloat16_rn(f.d2.y * a0.y));
          *reinterpret_cast<float2*>(a.kg + p * NK + i0) = a0;
        } else {
          const float2 z = a0;
          const Rbf2 f = rbf_eval2(z, s_r + i0 * RBF_LD, s_r + (i0 + 1) * RBF_LD);
          *reinterpret_cast<uint32_t*>(a.u + p * CU + i0) =
              pack2(__float2bfloat16_rn(f.d1.x), __float2bfloat16_rn(f.d1.y));
          *reinterpret_cast<float2*>(a.z + p * NK + i0) = z;
          if (NSRC == 2) {
            const float2 kg = make_float2(acc[NSRC - 1][r][nt][half * 2], acc[NSRC - 1][r][nt][half * 2 + 1]);
            *reinterpret_cast<uint32_t*>(a.v + p * CU + i0) =
                pack2(__float2bfloat16_rn(f.d2.x * kg.x), __float2bfloat16_rn(f.d2.y * kg.y));
            *reinterpret_cast<float2*>(a.kg + p * NK + i0) = kg;
          }
        }
      }
      // channels 24..31 of the stored activations are zero
      if (!ZIN) *reinterpret_cast<uint32_t*>(a.u + p * CU + NK + 2 * tig) = 0u;
      if (NSRC == 2 || ZIN) *reinterpret_cast<uint32_t*>(a.v + p * CU + NK + 2 * tig) = 0u;
    }
  }
}

// ------------------------------------------------- K (2 -> 24) on the tensor cores (tcgen05)
// One CTA per band of KC_R = 8 output rows x 128 pixels, as k_vn_K, with the contraction issued
// as tcgen05.mma (BF16 operands from shared memory, FP32 accumulators in tensor memory):
//   per source row s of the band (s - h0 = delta, -5 .. 12):
//     D[px][(r, i)] += sum_k A_s[px][k] B[(r, i)][k]   (M = 128 pixels, N = 8 rows x 32 filters, K = 80)
//   A_s = im2col of source row s: k = part * 24 + c * 11 + dx (three BF16 terms of x, as in k_vn_K;
//         columns 22, 23 of each part and 72 .. 79 zero);
//   B   = the filters of row dy = delta + 5 - r for output row r (zero outside 0 .. 10).  All eight
//         rows' blocks of one source row are a contiguous slice of one table: block j holds the
//         24 filters (8 zero rows) of filter row dy = 17 - j, j = 0 .. 24, and source row delta
//         takes blocks 12 - delta .. 19 - delta.
// Operands sit in shared memory in the no-swizzle K-major core-matrix layout: element (row, k) at
// (k / 8) * (rows * 16) + row * 16 + (k % 8) * 2 bytes (leading byte offset rows * 16 between the
// two 8-element K halves of one MMA, stride byte offset 128 between 8-row groups).  The im2col
// tile is double-buffered: thread 0 issues the five MMAs of a source row and commits them to the
// buffer's mbarrier; the tile is rebuilt only after the MMAs that read it two rows earlier have
// completed.  After the last source row the 8 warps read the accumulators (warp w: TMEM lanes of
// its quadrant w % 4, output rows 4 (w / 4) .. 4 (w / 4) + 3) and run the RBF epilogue of k_vn_K.
// Every wait is bounded; a CTA that gives up sets SENSE_STATUS_DEVICE_TIMEOUT (when a status word
// is given), drains its committed MMAs (bounded) and frees its tensor memory.
constexpr int KC_R = 8;
constexpr int KC_CHUNKS = 10;                          // K = 80: ten 8-element chunks (72 used)
constexpr int KC_A_CHUNK = TILE * 16;                  // bytes of one K chunk of the im2col tile
constexpr int KC_A_BYTES = KC_A_CHUNK * KC_CHUNKS;     // 20,480
constexpr int KC_NBLK = 25;                            // table blocks (filter rows dy = 17 - j)
constexpr int KC_BLK_BYTES = 32 * 16 * KC_CHUNKS;      // one block: 32 rows x 80 K = 5,120 bytes
constexpr int KC_B_BYTES = KC_NBLK * KC_BLK_BYTES;     // 128,000 (global table)
constexpr int KC_RING = 10;                            // blocks held in shared memory
constexpr int KC_RB_CHUNK = KC_RING * 32 * 16;         // one K chunk of the ring: 5,120 bytes
constexpr int KC_TMEM_COLS = 256;                      // 8 rows x 32 columns of FP32 accumulators

struct KcSmem {
  static constexpr int OFF_B = 0;                      // ring of KC_RING table blocks
  static constexpr int OFF_A = OFF_B + KC_RB_CHUNK * KC_CHUNKS;
  static constexpr int OFF_STG = OFF_A + 2 * KC_A_BYTES;
  static constexpr int OFF_PR = OFF_STG + 2 * K_STG * 8;
  static constexpr int PR_BYTES = K_PARTS * 2 * K_PR_LD * 2;
  static constexpr int OFF_R = OFF_PR + PR_BYTES;
  static constexpr int OFF_BAR = (OFF_R + NK * RBF_LD * 4 + 15) & ~15;
  static constexpr int TOTAL = OFF_BAR + 32;
};

// The K table, block-major: block j (32 rows, filter row dy = 17 - j) is contiguous, each of its
// K chunks a 512-byte core-matrix column (bf16 index j * 2560 + (k / 8) * 256 + f * 8 + k % 8).
__global__ void k_vn_pack_tc(const float* prm, bf16* wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= KC_NBLK * 32 * KC_CHUNKS * 8) return;
  const int n = i / (KC_CHUNKS * 8), k = i % (KC_CHUNKS * 8);
  const int j = n / 32, f = n % 32, dy = 17 - j;
  float v = 0.f;
  if (f < NK && dy >= 0 && dy < KS && k < K_KP && (k % 24) < 2 * KS) {
    const int kk = k % 24, c = kk / KS, dx = kk % KS;
    v = prm[(f * 2 + c) * NT + dy * KS + dx];
  }
  wt[(size_t)j * (KC_BLK_BYTES / 2) + (k / 8) * 256 + f * 8 + (k % 8)] = __float2bfloat16_rn(v);
}

template <bool ZIN>
__global__ void __launch_bounds__(K_THREADS, 2) k_vn_K_tc(const KArgs a, const bf16* wt, int* status) {
  using S = KcSmem;
  extern __shared__ __align__(16) uint8_t dsm[];
  float* s_r = reinterpret_cast<float*>(dsm + S::OFF_R);
  uint64_t* mma_done = reinterpret_cast<uint64_t*>(dsm + S::OFF_BAR);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(dsm + S::OFF_BAR + 16);
  int* s_err = reinterpret_cast<int*>(dsm + S::OFF_BAR + 20);
  const int w0 = blockIdx.x * TILE, h0 = blockIdx.y * KC_R, b = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    mbar_init(&mma_done[0], 1);
    mbar_init(&mma_done[1], 1);
    *s_err = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(s_tmem, KC_TMEM_COLS);
    tmem_relinquish();
  }
  // table block j into ring slot j % KC_RING (its K chunk kc: 32 rows x 16 bytes at kc * KC_RB_CHUNK)
  auto load_block = [&](int j) {
    const uint8_t* src = reinterpret_cast<const uint8_t*>(wt) + (size_t)j * KC_BLK_BYTES;
    uint8_t* dst = dsm + S::OFF_B + (j % KC_RING) * 512;
    for (int i = tid; i < KC_BLK_BYTES / 16; i += K_THREADS)
      cp16(dst + (i >> 5) * KC_RB_CHUNK + (i & 31) * 16, src + i * 16, true);
  };
  for (int i = tid; i < NK * RBF_LD; i += K_THREADS) {
    const int j = i % RBF_LD - RBF_PAD;
    s_r[i] = (unsigned)j < (unsigned)NW ? a.rbf[(i / RBF_LD) * NW + j] : 0.f;
  }
  const int s_lo = max(h0 - KH, 0), s_hi = min(h0 + KC_R - 1 + KH, a.H - 1);
  const int nrows = s_hi - s_lo + 1;
  auto stage = [&](int k) {
    const int s = s_lo + k, buf = k & 1;
    for (int q = tid; q < K_STG / 2; q += K_THREADS) {
      const int col = w0 - 6 + 2 * q;  // even; W is even, so col + 1 < W whenever col < W
      const bool ok = col >= 0 && col < a.W;
      cp16(dsm + S::OFF_STG + buf * K_STG * 8 + q * 16, a.x + (ok ? ((size_t)b * a.H + s) * a.W + col : 0), ok);
    }
  };
  // first source row: its x row and the eight table blocks of its window (12 - delta .. 19 - delta)
  const int jw0 = 12 - (s_lo - h0);
  for (int j = jw0; j < jw0 + KC_R; ++j) load_block(j);
  stage(0);
  cp_commit();
  // the unused last K chunk (k = 72 .. 79) of both im2col buffers is zero
  for (int i = tid; i < 2 * TILE; i += K_THREADS)
    *reinterpret_cast<uint4*>(dsm + S::OFF_A + (i / TILE) * KC_A_BYTES + 9 * KC_A_CHUNK + (i % TILE) * 16) =
        make_uint4(0u, 0u, 0u, 0u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  int last_issued = -1;  // thread 0: the last source row whose MMAs were committed

  // Source row k reads im2col buffer k & 1 and the ring slots of blocks j0 .. j0 + 7 (j0 = 12 -
  // delta, one less per row).  Before row k's x row and block j0 - 1 (for row k + 1) are copied in,
  // the MMAs of row k - 2 (the last reader of that buffer and of that slot: a ring of ten blocks)
  // must have completed.
#pragma unroll 1
  for (int k = 0; k < nrows; ++k) {
    const int j0 = 12 - (s_lo + k - h0);
    if (tid == 0 && k >= 2 && !mbar_wait(&mma_done[k & 1], ((k - 2) >> 1) & 1)) *s_err = 1;
    __syncthreads();
    if (*s_err) break;
    if (k + 1 < nrows) {
      stage(k + 1);
      load_block(j0 - 1);
    }
    cp_commit();
    cp_wait<1>();  // source row k and its window have landed
    __syncthreads();
    // BF16 terms of source row k
    for (int j = tid; j < K_STG; j += K_THREADS) {
      float2 v = reinterpret_cast<const float2*>(dsm + S::OFF_STG + (k & 1) * K_STG * 8)[j];
      bf16* pr = reinterpret_cast<bf16*>(dsm + S::OFF_PR);
#pragma unroll
      for (int part = 0; part < K_PARTS; ++part) {
        const bf16 re = __float2bfloat16_rn(v.x), im = __float2bfloat16_rn(v.y);
        pr[(part * 2) * K_PR_LD + j] = re;
        pr[(part * 2 + 1) * K_PR_LD + j] = im;
        v.x -= __bfloat162float(re);
        v.y -= __bfloat162float(im);
      }
    }
    __syncthreads();
    // im2col of source row k into buffer k & 1: item (part, pixel m) = 24 columns = 3 K chunks
    uint8_t* At = dsm + S::OFF_A + (k & 1) * KC_A_BYTES;
    for (int it = tid; it < K_PARTS * TILE; it += K_THREADS) {
      const int part = it / TILE, m = it % TILE;
      const uint32_t* r0 = reinterpret_cast<const uint32_t*>(dsm + S::OFF_PR + (part * 2) * K_PR_LD * 2);
      const uint32_t* r1 = r0 + K_PR_LD / 2;
      const int e0 = m + 1, w0i = e0 >> 1;
      const bool odd = e0 & 1;
      uint32_t A[6], Bw[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        A[q] = r0[w0i + q];
        Bw[q] = r1[w0i + q];
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        A[q] = odd ? __byte_perm(A[q], A[q + 1], 0x5432) : A[q];
        Bw[q] = odd ? __byte_perm(Bw[q], Bw[q + 1], 0x5432) : Bw[q];
      }
      A[5] = odd ? (A[5] >> 16) : (A[5] & 0xffffu);
      Bw[5] = odd ? (Bw[5] >> 16) : (Bw[5] & 0xffffu);
      uint8_t* dst = At + (part * 3) * KC_A_CHUNK + m * 16;
      *reinterpret_cast<uint4*>(dst) = make_uint4(A[0], A[1], A[2], A[3]);
      *reinterpret_cast<uint4*>(dst + KC_A_CHUNK) =
          make_uint4(A[4], A[5] | (Bw[0] << 16), __byte_perm(Bw[0], Bw[1], 0x5432), __byte_perm(Bw[1], Bw[2], 0x5432));
      *reinterpret_cast<uint4*>(dst + 2 * KC_A_CHUNK) =
          make_uint4(__byte_perm(Bw[2], Bw[3], 0x5432), __byte_perm(Bw[3], Bw[4], 0x5432),
                     __byte_perm(Bw[4], Bw[5], 0x5432), 0u);
    }
    fence_proxy_async();  // this thread's shared-memory writes (and landed copies) -> tensor core
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      // the window's 256 rows start at ring slot j0 % KC_RING; where they wrap past the last slot
      // the MMA is split in two (N1 + N2 = 256 accumulator columns, both multiples of 32)
      const int sl = j0 % KC_RING;
      const int n1 = min(KC_RING - sl, KC_R) * 32, n2 = KC_R * 32 - n1;
      const uint32_t sa = smem_u32(At), sb = smem_u32(dsm + S::OFF_B);
      const uint32_t id1 = umma_idesc_bf16(TILE, n1), id2 = umma_idesc_bf16(TILE, n2 > 0 ? n2 : 32);
#pragma unroll
      for (int ks = 0; ks < 5; ++ks) {
        const uint64_t ad = umma_desc(sa + ks * 2 * KC_A_CHUNK, KC_A_CHUNK, 128);
        const uint32_t bk = sb + ks * 2 * KC_RB_CHUNK;
        umma_bf16(tmem, ad, umma_desc(bk + sl * 512, KC_RB_CHUNK, 128), id1, (k | ks) != 0);
        if (n2 > 0) umma_bf16(tmem + n1, ad, umma_desc(bk, KC_RB_CHUNK, 128), id2, (k | ks) != 0);
      }
      umma_commit(&mma_done[k & 1]);
      last_issued = k;
    }
  }
  // accumulators of the band: every lane waits for the last commit
  bool ok = *s_err == 0;
  if (ok) {
    const int kl = nrows - 1;
    const bool got = mbar_wait(&mma_done[kl & 1], (kl >> 1) & 1);
    if (!got) atomicExch(s_err, 1);
    ok = __all_sync(0xffffffffu, got);
  }
  tc_fence_after();
  if (ok) {
    const int q = warp & 3;
    const int w = w0 + q * 32 + lane;
#pragma unroll 1
    for (int rr = 0; rr < 4; ++rr) {
      const int r = (warp >> 2) * 4 + rr, h = h0 + r;
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
      float acc[16];
      __syncwarp();  // the TMEM loads are warp-collective
      tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + r * 32 + half * 16, acc);
      if (h >= a.H || w >= a.W) continue;
      const size_t p = ((size_t)b * a.H + h) * a.W + w;
#pragma unroll
      for (int e = 0; e < 16; e += 2) {
        const int i0 = half * 16 + e;
        if (i0 >= NK) break;
        const float2 a0 = make_float2(acc[e], acc[e + 1]);
        if constexpr (ZIN) {  // a0 = K g; z from the forward stage
          const float2 z = *reinterpret_cast<const float2*>(a.z + p * NK + i0);
          const Rbf2 f = rbf_eval2(z, s_r + i0 * RBF_LD, s_r + (i0 + 1) * RBF_LD);
          *reinterpret_cast<uint32_t*>(a.v + p * CU + i0) =
              pack2(__float2bfloat16_rn(f.d2.x * a0.x), __float2bfloat16_rn(f.d2.y * a0.y));
          *reinterpret_cast<float2*>(a.kg + p * NK + i0) = a0;
        } else {
          const Rbf2 f = rbf_eval2(a0, s_r + i0 * RBF_LD, s_r + (i0 + 1) * RBF_LD);
          *reinterpret_cast<uint32_t*>(a.u + p * CU + i0) =
              pack2(__float2bfloat16_rn(f.d1.x), __float2bfloat16_rn(f.d1.y));
          *reinterpret_cast<float2*>(a.z + p * NK + i0) = a0;
        }
      }
      // channels 24..31 of the stored activations are zero
      if (half == 1) *reinterpret_cast<uint4*>((ZIN ? a.v : a.u) + p * CU + NK) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*s_err && tid == 0) {
    if (status) set_status(status, SENSE_STATUS_DEVICE_TIMEOUT);
    if (last_issued >= 0) mbar_wait(&mma_done[last_issued & 1], (last_issued >> 1) & 1, 1u << 20);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, KC_TMEM_COLS);
}

// ------------------------------------------------------------ K^T (24 -> 2)
// out = base + sgn K^T(src) - lambda (n - c): base, n and c may be NULL (zero; no data term
// without n)
// CTA: 128 pixels x 8 output rows, 4 warps x 32 pixels.  For source row s and tap column dx:
//   D[px][(r, c)] += sum_i src[s][px + 5 - dx][i] w[i][c][h0 + r + 5 - s][dx]
// (A = the staged source row via ldmatrix, B = the filter taps of the two output channels for
// output rows r = 0..3 and 4..7, zero where the filter row falls outside 0..10).
struct KTArgs {
  int B, H, W;
  const bf16* src;  // [px][32]
  const bf16* wn;   // [11][11][2][KT_LDW]
  const float2* base;
  const float2* n;
  const float2* c;
  const float* lam;
  float sgn;
  float2* out;
};

constexpr int KT_BAND = 8;
constexpr int KT_NBUF = 3;
constexpr int KT_ROW = HW_ * LDI;  // bf16 elements of one staged source row
constexpr int KT_W_BYTES = KT_W_ELEMS * 2;
constexpr int KT_SMEM = KT_W_BYTES + KT_NBUF * KT_ROW * 2;

__global__ void __launch_bounds__(128, 4) k_vn_KT(const KTArgs a) {
  extern __shared__ __align__(16) uint8_t dsm[];
  const bf16* wn = reinterpret_cast<const bf16*>(dsm);
  bf16* ub = reinterpret_cast<bf16*>(dsm + KT_W_BYTES);
  const int w0 = blockIdx.x * TILE, h0 = blockIdx.y * KT_BAND, b = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gid = lane >> 2, tig = lane & 3, mi = lane >> 3, rr = lane & 7;
  for (int i = tid; i < KT_W_BYTES / 16; i += blockDim.x)
    cp16(dsm + i * 16, reinterpret_cast<const uint8_t*>(a.wn) + i * 16, true);
  const int s_lo = max(h0 - KH, 0), s_hi = min(h0 + KT_BAND - 1 + KH, a.H - 1);
  const int nrows = s_hi - s_lo + 1;
  auto stage = [&](int k) {
    const int s = s_lo + k;
    bf16* dst = ub + (k % KT_NBUF) * KT_ROW;
    for (int i = tid; i < HW_ * 4; i += blockDim.x) {
      const int px = i >> 2, q = i & 3;
      const int xx = w0 - KH + px;
      const bool ok = xx >= 0 && xx < a.W;
      cp16(dst + px * LDI + q * 8, a.src + (ok ? (((size_t)b * a.H + s) * a.W + xx) * CU + q * 8 : 0), ok);
    }
  };
  stage(0);
  cp_commit();
  if (nrows > 1) stage(1);
  cp_commit();
  float d[2][2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) d[mt][nt][e] = 0.f;

#pragma unroll 1
  for (int k = 0; k < nrows; ++k) {
    cp_wait<1>();  // source row k has landed (only row k + 1 may be pending)
    __syncthreads();  // ... for every thread; and row k - 1's buffer is free for row k + 2
    if (k + 2 < nrows) stage(k + 2);
    cp_commit();
    const int s = s_lo + k;
    const bf16* u = ub + (k % KT_NBUF) * KT_ROW;
    const bool v0 = s >= h0 - KH && s <= h0 + 3 + KH;  // some output row 0..3 uses source row s
    const bool v1 = s >= h0 + 4 - KH && s <= h0 + 7 + KH;
#pragma unroll 1
    for (int dx = 0; dx < KS; ++dx) {
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        uint32_t bq[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int r = nt * 4 + (gid >> 1), c = gid & 1, dy = h0 + r + KH - s;
          bq[nt][0] = bq[nt][1] = 0u;
          if ((unsigned)dy < (unsigned)KS) {
            const bf16* wp = wn + ((dy * KS + dx) * 2 + c) * KT_LDW + ks * 16 + 2 * tig;
            bq[nt][0] = *reinterpret_cast<const uint32_t*>(wp);
            bq[nt][1] = *reinterpret_cast<const uint32_t*>(wp + 8);
          }
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          uint32_t af[4];
          const int m = warp * 32 + mt * 16 + (mi & 1) * 8 + rr;
          ldsm4(af, u + (m + 2 * KH - dx) * LDI + ks * 16 + (mi >> 1) * 8);
          if (v0) mma16816(d[mt][0], af, bq[0][0], bq[0][1]);
          if (v1) mma16816(d[mt][1], af, bq[1][0], bq[1][1]);
        }
      }
    }
  }
  // epilogue: (c0, c1) = (re, im) of pixel gid, output row nt * 4 + tig; (c2, c3) pixel gid + 8
  const float lam = a.n ? a.lam[0] : 0.f;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int h = h0 + nt * 4 + tig;
      if (h >= a.H) continue;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int w = w0 + warp * 32 + mt * 16 + gid + half * 8;
        if (w >= a.W) continue;
        const size_t p = ((size_t)b * a.H + h) * a.W + w;
        float2 o = make_float2(a.sgn * d[mt][nt][2 * half], a.sgn * d[mt][nt][2 * half + 1]);
        if (a.base) {
          const float2 bv = a.base[p];
          o.x += bv.x;
          o.y += bv.y;
        }
        if (a.n) {
          const float2 nv = a.n[p];
          const float2 cv = a.c ? a.c[p] : make_float2(0.f, 0.f);
          o.x -= lam * (nv.x - cv.x);
          o.y -= lam * (nv.y - cv.y);
        }
        a.out[p] = o;
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

// RBF weight gradient partial per image row: P[i][j] = sum_w kg[w][i] phi_j(z[w][i]).
// Thread (i, q), i < 24, q < 10, takes pixels w = q, q + 10, ... and adds into its own
// shared-memory row of 31 accumulators (13-centre window by the product recurrence of
// rbf_eval2); the ten rows of each filter are then added in order.
constexpr int RG_Q = 10;
__global__ void __launch_bounds__(256) k_vn_rbfgrad(int B, int H, int W, const float* z, const float* kg,
                                                    float* partial) {
  // accumulator j of thread t at acc[j * 256 + t]: every thread keeps to its own bank whatever
  // window its pixel's z selects (a thread-major layout put the lanes of a warp on banks that
  // depend on z, and the read-modify-writes conflicted)
  __shared__ float acc[NW * 256];
  const int t = threadIdx.x;
  for (int k = t; k < NW * 256; k += blockDim.x) acc[k] = 0.f;
  __syncthreads();
  const int b = blockIdx.x / H, h = blockIdx.x % H;
  if (t < NK * RG_Q) {
    const int i = t % NK, q = t / NK;
    float* my = acc + t;
    for (int w = q; w < W; w += RG_Q) {
      const size_t p = ((size_t)b * H + h) * W + w;
      const float zz = z[p * NK + i], g = kg[p * NK + i];
      float d;
      const int j0 = window_start(zz, d);
      float phi = zz == zz ? g * expf(-0.5f * d * d) : zz;  // NaN propagates
      float rho = expf(d - 0.5f);
#pragma unroll
      for (int k = 0; k < RBF_WIN; ++k) {
        if ((unsigned)(j0 + k) < (unsigned)NW) my[(j0 + k) * 256] += phi;
        phi *= rho;
        rho *= kEinv;
      }
    }
  }
  __syncthreads();
  float* out = partial + (size_t)blockIdx.x * (NK * NW);
  for (int k = t; k < NK * NW; k += blockDim.x) {
    const int i = k / NW, j = k % NW;
    float s = 0.f;
    for (int q = 0; q < RG_Q; ++q) s += acc[j * 256 + q * NK + i];
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

size_t up256(size_t n) { return (n + 255) & ~(size_t)255; }

struct VnLayout {
  size_t wk, wn, wtc, u, v, z, kg, n1, n2, part, part2, pdot, total;
};
VnLayout vn_layout(int B, int H, int W) {
  VnLayout L;
  const size_t px = (size_t)B * H * W;
  size_t o = 0;
  L.wk = o; o += up256(K_W_ELEMS * 2);
  L.wn = o; o += up256(KT_W_ELEMS * 2);
  L.wtc = o; o += up256(KC_B_BYTES);
  L.u = o; o += up256(px * CU * 2);
  L.v = o; o += up256(px * CU * 2);
  L.z = o; o += up256(px * NK * 4);
  L.kg = o; o += up256(px * NK * 4);
  L.n1 = o; o += up256(px * 8);
  L.n2 = o; o += up256(px * 8);
  L.part = o; o += up256((size_t)B * H * NK * 2 * NT * 4);  // filter-gradient rows
  L.part2 = o; o += up256((size_t)B * H * NK * NW * 4);     // RBF-gradient rows (run beside them)
  L.pdot = o; o += 256;
  L.total = o;
  return L;
}

int vn_prepare() {
  static int state = 0;
  static std::mutex mu;
  std::lock_guard<std::mutex> l(mu);
  if (state == 0)
    state = (             cudaFuncSetAttribute(k_vn_K_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, KcSmem::TOTAL) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(k_vn_K_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, KcSmem::TOTAL) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(k_vn_K<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, KSmem<2>::TOTAL) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(k_vn_KT, cudaFuncAttributeMaxDynamicSharedMemorySize, KT_SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_vn_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, wg_smem(WG_MAXW)) ==
                 cudaSuccess)
                ? 1
                : -1;
  return state == 1 ? SENSE_OK : SENSE_ECUDA;
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int vn_shape_check(int B, int H, int W) {
  if (B <= 0 || H <= 0 || W <= 0 || (W & 1)) return SENSE_EINVAL_SHAPE;
  if (W > WG_MAXW || B > 65535 || (H + 3) / 4 > 65535) return SENSE_EUNSUPPORTED;
  return SENSE_OK;
}

int vn_check(sense_plan p, const float* prm, const void* AHy, const void* xt, const void* nx, void* ws,
             size_t ws_bytes) {
  if (!p || !prm || !AHy || !xt || !ws || !al16(AHy) || !al16(xt) || (nx && !al16(nx)) || ((uintptr_t)ws & 255u))
    return SENSE_EINVAL_PTR;
  if (int e = vn_shape_check(p->B, p->H, p->W)) return e;
  if (p->S != 1) return SENSE_EUNSUPPORTED;  // one image per slice
  if (ws_bytes < vn_layout(p->B, p->H, p->W).total) return SENSE_EWORKSPACE;
  return vn_prepare();
}

struct Shape {
  int B, H, W;
  cudaStream_t st;
  int* status = nullptr;  // device status word for bounded-wait timeouts (plan calls), or none
};

void vn_pack(const float* prm, uint8_t* ws, const VnLayout& L, cudaStream_t st) {
  const int n = K_W_ELEMS + KT_W_ELEMS;
  prof_mark("vn_misc", st, false);
  k_vn_pack<<<(n + 255) / 256, 256, 0, st>>>(prm, reinterpret_cast<bf16*>(ws + L.wk),
                                             reinterpret_cast<bf16*>(ws + L.wn));
  const int ntc = KC_NBLK * 32 * KC_CHUNKS * 8;
  k_vn_pack_tc<<<(ntc + 255) / 256, 256, 0, st>>>(prm, reinterpret_cast<bf16*>(ws + L.wtc));
  prof_mark("vn_misc", st, true);
}

// nsrc 1: forward (z, u from x); 2: reverse recomputing z (z, u, kg, v from x and g); 3: reverse
// with z and u kept by the forward stage (kg, v from g alone)
int launch_K(const Shape& sh, int nsrc, const float* prm, const float2* x, const float2* g, uint8_t* ws,
             const VnLayout& L) {
  KArgs a;
  a.B = sh.B; a.H = sh.H; a.W = sh.W;
  a.x = nsrc == 3 ? g : x; a.g = g;
  a.wk = reinterpret_cast<const bf16*>(ws + L.wk);
  a.rbf = prm + OFF_RBF;
  a.u = reinterpret_cast<bf16*>(ws + L.u);
  a.v = reinterpret_cast<bf16*>(ws + L.v);
  a.z = reinterpret_cast<float*>(ws + L.z);
  a.kg = reinterpret_cast<float*>(ws + L.kg);
  const int R = nsrc == 2 ? K_RMAX / 2 : KC_R;
  const dim3 grid((sh.W + TILE - 1) / TILE, (sh.H + R - 1) / R, sh.B);
  const char* grp = nsrc >= 2 ? "vn_Kbwd" : "vn_K";
  const bf16* wtc = reinterpret_cast<const bf16*>(ws + L.wtc);
  prof_mark(grp, sh.st, false);
  if (nsrc == 2)  // K x and K g together (the recomputing reverse pass): warp-level tensor cores
    k_vn_K<2><<<grid, K_THREADS, KSmem<2>::TOTAL, sh.st>>>(a);
  else if (nsrc == 3)
    k_vn_K_tc<true><<<grid, K_THREADS, KcSmem::TOTAL, sh.st>>>(a, wtc, sh.status);
  else
    k_vn_K_tc<false><<<grid, K_THREADS, KcSmem::TOTAL, sh.st>>>(a, wtc, sh.status);
  prof_mark(grp, sh.st, true);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int launch_KT(const Shape& sh, const bf16* src, const float* prm, float sgn, const float2* base,
              const float2* n, const float2* c, float2* out, uint8_t* ws, const VnLayout& L) {
  KTArgs a;
  a.B = sh.B; a.H = sh.H; a.W = sh.W;
  a.src = src;
  a.wn = reinterpret_cast<const bf16*>(ws + L.wn);
  a.base = base; a.n = n; a.c = c; a.lam = prm + OFF_LAM; a.sgn = sgn; a.out = out;
  const dim3 grid((sh.W + TILE - 1) / TILE, (sh.H + KT_BAND - 1) / KT_BAND, sh.B);
  prof_mark("vn_KT", sh.st, false);
  k_vn_KT<<<grid, 128, KT_SMEM, sh.st>>>(a);
  prof_mark("vn_KT", sh.st, true);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

// Parameter gradients of the regulariser sum_i K_i^T Phi_i'(K_i x), scaled by `scale` and added to
// grad_prm: filters  scale * sum (u (x) g_shift + v (x) x_shift),  RBF weights  scale * sum kg phi_j(z).
// Needs u, v, z, kg of a two-source K launch in the workspace.
// The filter gradient runs on stream s_w and the RBF-weight gradient on s_r (the same stream or
// two side streams: they read the workspace and write disjoint parts of grad_prm).
void launch_param_grads(const Shape& sh, const float2* x, const float2* g, float scale, float* grad_prm,
                        uint8_t* ws, const VnLayout& L, cudaStream_t s_w, cudaStream_t s_r) {
  const int rows = sh.B * sh.H;
  float* part = reinterpret_cast<float*>(ws + L.part);
  float* part2 = reinterpret_cast<float*>(ws + L.part2);
  prof_mark("vn_wgrad", s_w, false);
  k_vn_wgrad<<<rows, 128, wg_smem(sh.W), s_w>>>(sh.B, sh.H, sh.W, reinterpret_cast<const bf16*>(ws + L.u),
                                                 reinterpret_cast<const bf16*>(ws + L.v), g, x, part);
  k_vn_reduce<<<(NK * 2 * NT + 31) / 32, 256, 0, s_w>>>(part, rows, NK * 2 * NT, scale, grad_prm);
  prof_mark("vn_wgrad", s_w, true);
  prof_mark("vn_rbfgrad", s_r, false);
  k_vn_rbfgrad<<<rows, 256, 0, s_r>>>(sh.B, sh.H, sh.W, reinterpret_cast<const float*>(ws + L.z),
                                       reinterpret_cast<const float*>(ws + L.kg), part2);
  k_vn_reduce<<<(NK * NW + 31) / 32, 256, 0, s_r>>>(part2, rows, NK * NW, scale, grad_prm + OFF_RBF);
  prof_mark("vn_rbfgrad", s_r, true);
}

// Normal operator without lambda (A^H A x) through the plan's own path, on stream s (the plan's
// stream is switched for the call; a plan is used by one host thread at a time).
int normal0(sense_plan p, const float2* x, float2* out, cudaStream_t s) {
  const cudaStream_t own = p->stream;
  p->stream = s;
  const int e = sense_normal(p, x, out, 0.f);
  p->stream = own;
  return e;
}

// d/dlambda of the stage: -Re<g, n - c>, added to grad[OFF_LAM] (float32).
__global__ void k_vn_addlam(const double* d, float* g) { g[OFF_LAM] += (float)(-d[0]); }

}  // namespace

extern "C" {

size_t varnet_workspace_bytes(int B, int H, int W) {
  if (B <= 0 || H <= 0 || W <= 0) return 0;
  return vn_layout(B, H, W).total;
}

int varnet_param_count(void) { return NPAR; }

int varnet_workspace_offsets(int B, int H, int W, size_t* offsets) {
  if (B <= 0 || H <= 0 || W <= 0) return SENSE_EINVAL_SHAPE;
  if (!offsets) return SENSE_EINVAL_PTR;
  const VnLayout L = vn_layout(B, H, W);
  offsets[0] = L.u;
  offsets[1] = L.v;
  offsets[2] = L.z;
  offsets[3] = L.kg;
  return SENSE_OK;
}

int varnet_stage(sense_plan p, const float* prm, const void* AHy, const void* x_t, void* x_next, void* nx_out,
                 void* ws, size_t ws_bytes) {
  if (int e = vn_check(p, prm, AHy, x_t, nx_out, ws, ws_bytes)) return e;
  if (!x_next || !al16(x_next) || x_next == x_t || nx_out == x_t || nx_out == x_next) return SENSE_EINVAL_PTR;
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  const VnLayout L = vn_layout(p->B, p->H, p->W);
  const Shape sh{p->B, p->H, p->W, p->stream, p->status};
  const float2* x = static_cast<const float2*>(x_t);
  float2* n1 = nx_out ? static_cast<float2*>(nx_out) : reinterpret_cast<float2*>(w8 + L.n1);
  // A^H A x on a side stream beside z = K x and u = Phi'(z); both feed the combine
  SideSet* ss = nullptr;
  if (int e = side_set(&ss)) return e;
  const cudaStream_t sd = ss->s[1];
  if (int e = stream_after(*ss, p->stream, sd)) return e;
  if (int e = normal0(p, x, n1, sd)) return e;
  vn_pack(prm, w8, L, p->stream);
  if (int e = launch_K(sh, 1, prm, x, nullptr, w8, L)) return e;
  if (int e = stream_after(*ss, sd, p->stream)) return e;
  if (int e = launch_KT(sh, reinterpret_cast<const bf16*>(w8 + L.u), prm, -1.f, x, n1,
                        static_cast<const float2*>(AHy), static_cast<float2*>(x_next), w8, L))
    return e;
  prof_count(3);
  return SENSE_OK;
}

int varnet_stage_backward_ex(sense_plan p, const float* prm, const void* AHy, const void* x_t, const void* nx_t,
                             const void* grad_next, void* grad_t, float* grad_prm, void* ws, size_t ws_bytes,
                             int recompute) {
  if (int e = vn_check(p, prm, AHy, x_t, nx_t, ws, ws_bytes)) return e;
  if (!grad_next || !grad_t || !grad_prm || !al16(grad_next) || !al16(grad_t) || grad_t == grad_next ||
      grad_t == nx_t)
    return SENSE_EINVAL_PTR;
  if (!p->ws) return SENSE_EWORKSPACE;  // the lambda-gradient dot uses the plan's workspace
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  const VnLayout L = vn_layout(p->B, p->H, p->W);
  const Shape sh{p->B, p->H, p->W, p->stream, p->status};
  const float2* x = static_cast<const float2*>(x_t);
  const float2* g = static_cast<const float2*>(grad_next);
  float2* n2 = reinterpret_cast<float2*>(w8 + L.n2);
  double* pdot = reinterpret_cast<double*>(w8 + L.pdot);
  vn_pack(prm, w8, L, p->stream);
  // grad lambda_t = -Re<g, A^H A x - A^H y>  (A^H A x from the forward when given)
  const float2* n1 = static_cast<const float2*>(nx_t);
  if (!n1) {
    float2* t = reinterpret_cast<float2*>(w8 + L.n1);
    if (int e = normal0(p, x, t, p->stream)) return e;
    n1 = t;
  }
  if (int e = launch_dot_rows(p, g, n1, static_cast<const float2*>(AHy), pdot, 1, 0)) return e;
  prof_mark("vn_misc", p->stream, false);
  k_vn_addlam<<<1, 1, 0, p->stream>>>(pdot, grad_prm);
  prof_mark("vn_misc", p->stream, true);
  // Side streams: the filter gradient runs on s0 and the RBF-weight gradient on s1; A^H A g runs
  // on s1 before it (joined calls) or alone on s2 (deferred calls, whose gradients are not joined:
  // the next stage's A^H A g then does not queue behind them; sense_streams_join ends them).
  // The caller's stream runs K g and the combine.
  const bool defer = (recompute & SENSE_VN_DEFER_JOIN) != 0;
  recompute &= 1;
  SideSet* ss = nullptr;
  if (int e = side_set(&ss)) return e;
  const cudaStream_t s0 = ss->s[0], s1 = ss->s[1], sn = defer ? ss->s[2] : ss->s[1];
  if (int e = stream_after(*ss, p->stream, sn)) return e;
  if (int e = normal0(p, g, n2, sn)) return e;
  // z = K x (recomputed, or kept in ws by this stage's forward together with u = Phi'(z)), kg = K g,
  // v = Phi''(z) kg; parameter gradients of -R beside the combine (they read g, x, u, v, z, kg)
  if (int e = launch_K(sh, recompute ? 2 : 3, prm, x, g, w8, L)) return e;
  if (defer) {
    if (int e = stream_after(*ss, sn, p->stream)) return e;  // A^H A g done
    if (int e = stream_after(*ss, p->stream, s0)) return e;
    if (int e = stream_after(*ss, p->stream, s1)) return e;
    launch_param_grads(sh, x, g, -1.f, grad_prm, w8, L, s0, s1);
  } else {
    if (int e = stream_after(*ss, p->stream, s0)) return e;
    if (int e = stream_after(*ss, p->stream, s1)) return e;
    launch_param_grads(sh, x, g, -1.f, grad_prm, w8, L, s0, s1);
    if (int e = stream_after(*ss, s1, p->stream)) return e;  // A^H A g and the RBF gradient done
  }
  // grad_t = g - K^T v - lambda A^H A g
  if (int e = launch_KT(sh, reinterpret_cast<const bf16*>(w8 + L.v), prm, -1.f, g, n2, nullptr,
                        static_cast<float2*>(grad_t), w8, L))
    return e;
  if (!defer)
    if (int e = stream_after(*ss, s0, p->stream)) return e;
  prof_count(8);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int varnet_stage_backward(sense_plan p, const float* prm, const void* AHy, const void* x_t, const void* nx_t,
                          const void* grad_next, void* grad_t, float* grad_prm, void* ws, size_t ws_bytes) {
  return varnet_stage_backward_ex(p, prm, AHy, x_t, nx_t, grad_next, grad_t, grad_prm, ws, ws_bytes, 1);
}

}  // extern "C"

// The regulariser R(x) = sum_i K_i^T Phi_i'(K_i x) alone, as the VarNet kind of the denoiser calls.
size_t vn_denoiser_bytes(int B, int H, int W) {
  if (vn_shape_check(B, H, W)) return 0;
  return vn_layout(B, H, W).total;
}

int vn_denoiser_forward(const float* prm, const void* x, void* out, void* ws, size_t ws_bytes, int B, int H, int W,
                        cudaStream_t st) {
  if (int e = vn_shape_check(B, H, W)) return e;
  if (!prm || !x || !out || !ws || !al16(x) || !al16(out) || x == out || ((uintptr_t)ws & 255u))
    return SENSE_EINVAL_PTR;
  const VnLayout L = vn_layout(B, H, W);
  if (ws_bytes < L.total) return SENSE_EWORKSPACE;
  if (int e = vn_prepare()) return e;
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  const Shape sh{B, H, W, st};
  vn_pack(prm, w8, L, st);
  if (int e = launch_K(sh, 1, prm, static_cast<const float2*>(x), nullptr, w8, L)) return e;
  if (int e = launch_KT(sh, reinterpret_cast<const bf16*>(w8 + L.u), prm, 1.f, nullptr, nullptr, nullptr,
                        static_cast<float2*>(out), w8, L))
    return e;
  prof_count(3);
  return SENSE_OK;
}

int vn_denoiser_backward(const float* prm, const void* x, const void* grad_out, void* grad_x, float* grad_prm,
                         void* ws, size_t ws_bytes, int B, int H, int W, cudaStream_t st) {
  if (int e = vn_shape_check(B, H, W)) return e;
  if (!prm || !x || !grad_out || !grad_x || !grad_prm || !ws || !al16(x) || !al16(grad_out) || !al16(grad_x) ||
      grad_x == grad_out || ((uintptr_t)ws & 255u))
    return SENSE_EINVAL_PTR;
  const VnLayout L = vn_layout(B, H, W);
  if (ws_bytes < L.total) return SENSE_EWORKSPACE;
  if (int e = vn_prepare()) return e;
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  const Shape sh{B, H, W, st};
  const float2* xx = static_cast<const float2*>(x);
  const float2* g = static_cast<const float2*>(grad_out);
  vn_pack(prm, w8, L, st);
  if (int e = launch_K(sh, 2, prm, xx, g, w8, L)) return e;
  launch_param_grads(sh, xx, g, 1.f, grad_prm, w8, L, st, st);
  // dR/dx^H g = K^T (Phi''(K x) K g)  (the Jacobian of R is symmetric)
  if (int e = launch_KT(sh, reinterpret_cast<const bf16*>(w8 + L.v), prm, 1.f, nullptr, nullptr, nullptr,
                        static_cast<float2*>(grad_x), w8, L))
    return e;
  prof_count(6);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}
