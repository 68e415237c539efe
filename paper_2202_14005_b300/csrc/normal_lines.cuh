// Fused SENSE normal operator for Cartesian line masks (hot path).
//
//   out = sum_c conj(S_c) * F^{-1} M^2 F (S_c * x) + lambda * x      (Eq. 4, Eq. 6)
//
// With a mask constant along H (phase-encode lines along W), the 2-D transform
// reduces row by row: F^{-1} diag(m) F = I_H (x) (F_W^{-1} diag(m) F_W), since the
// H-direction transform meets its own inverse.  The centring of the unitary DFT
// cancels as well (F_W^{-1} diag(m) F_W is circulant), leaving a plain DFT pair
// with the mask shifted to plain frequency order and a 1/W scale.
//
// Each row-coil pair is transformed with W = Q * P (Q a power of two):
//   phase A  lane t < P holds u[t + P n1], n1 < Q: Q-point DFT in registers,
//            twiddle by e^{-2 pi i t k1 / W}, store to shared memory as [k1][t];
//   phase B  lane (coil gi, residue k1): the P-point DFT over t is evaluated only
//            at the sampled frequencies k = k1 + Q k2 (pruned, using the pairing
//            t <-> P - t), weighted by mask^2 / W, and transformed back (again
//            only from the sampled frequencies) — no coil image or k-space ever
//            leaves the SM;
//   phase C  inverse twiddle, inverse Q-point DFT in registers, accumulate
//            conj(S_c) * v over the coils of the warp.
// Warps of one row sum their coil groups through shared memory in a fixed
// order; per-row partials of the CG inner products are written (FP32 lane sums
// carried across lanes and warps as float-float pairs), and the last CTA to
// finish reduces them per slice (fixed order, deterministic).
#pragma once
#include <algorithm>
#include <cmath>

#include "plan.cuh"

// Kernel template and its launch arguments; the instantiations live in normal_lines_q8.cu and
// normal_lines_q16.cu (compiled in parallel), the tables and the launcher in normal_lines.cu.
namespace nl {

struct NLArgs {
  int B, C, H, HS, J, kstride, rows, nwr, tiles_per_slice, ntiles;  // HS = sets * H (CG rows per slice)
  const float2* maps;
  const float4* coef;
  const float2* tw;
  const float* wt;
  const float* sgn;
  const int* akx;   // NM_ADJ: centred column of slot (k1, j)
  const float* af;  // NM_ADJ: slot factor (-1)^k / sqrt(W)
  const float2* x;  // NM_ADJ: column-transformed k-space T [B][C][H][W]; NM_CG2: r
  // NM_CG2 (one pass of the single-reduction CG): with upd, first p = r + beta p, s = w + beta s
  // (p = r, s = w when first), x += alpha p, r -= alpha s; then w = S r; rows of Re<r, w> to part
  // and of ||r||^2 to part2.  alpha, beta per slice (shared memory of the solve kernel).
  float2* sv = nullptr;
  float2* xs = nullptr;
  double* part2 = nullptr;
  const float* ab_f = nullptr;  // NM_CG2: alpha, beta of the tile's slice
  int upd = 0, first = 0;
  const float2* rhs0 = nullptr;  // NM_CG2 without upd: stage r = rhs0 (written to r) and zero x
  const float2* rhs0b = nullptr;  // with rhs0: r = rhs0 + lambda rhs0b (the MoDL right-hand side)
  const float2* pold;
  float2* pout;
  float2* out;
  const float2* rhs;
  float lam_host;
  const double* lam_dev;
  int lam_shared = 0;  // lam_dev holds one value for every slice (else one per slice)
  const double* beta;
  double* part;
  int finalize;
  double* rr;
  double* alpha;
  double* rr_hist_row;
  unsigned* counter;
  int* status;
};

// Shared-memory layout (bytes), identical on host and device.
struct NLLayout {
  int coef, tw, wt, sgn, x, y, total;
};
SENSE_HD NLLayout nl_layout(int Q, int P, int J, int kstride, int rows, int nwarps, int GB, int NS) {
  NLLayout L;
  const int W = Q * P;
  L.coef = 0;
  L.tw = L.coef + Q * kstride * 16;
  L.wt = L.tw + Q * P * 8;
  L.sgn = L.wt + Q * J * 4;
  L.x = (L.sgn + Q * J * 4 + 15) & ~15;
  L.y = L.x + NS * rows * W * 8;
  L.total = L.y + nwarps * GB * W * 8;
  return L;
}

// Fixed-order per-slice reductions done by the last CTA of a launch.
__device__ inline void nl_finalize(const NLArgs& a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int b = warp; b < a.B; b += nwarps) {
    double s = lane_strided_sum(a.part + (size_t)b * a.HS, a.HS, lane);
    s = warp_sum_d(s);
    if (lane != 0) continue;
    if (a.finalize == 1) {  // alpha = ||r||^2 / Re<p, S p>
      const double rr = __ldcg(a.rr + b);
      double al = 0.0;
      if (!isfinite(s) || !isfinite(rr)) set_status(a.status, SENSE_DEVST_NONFINITE);
      else if (rr > 0.0) {
        if (s > 0.0) al = rr / s;
        else set_status(a.status, SENSE_DEVST_CG_BREAKDOWN);
      }
      a.alpha[b] = al;
    } else {  // initial residual norm
      if (!isfinite(s)) set_status(a.status, SENSE_DEVST_NONFINITE);
      a.rr[b] = s;
      if (a.rr_hist_row) a.rr_hist_row[b] = s;
    }
  }
}

__device__ inline void last_block(const NLArgs& a) {
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
    nl_finalize(a);
    __syncthreads();
    if (threadIdx.x == 0) *a.counter = 0u;
  }
}

#define NL_CONSTS                                                                          \
  constexpr int GB = 32 / Q;          /* coils per warp in phase B */                         \
  constexpr int GA = 32 / P;          /* coils per pass in phases A/C */                      \
  constexpr int HP = (P - 1) / 2;     /* conjugate pairs t <-> P - t, t = 1..HP */            \
  constexpr bool EVENP = (P % 2) == 0;                                                         \
  constexpr int RQ = (HP + 1) / 2;    /* float4 quads per slot row */                         \
  constexpr int W = Q * P;                                                                     \
  constexpr int NPASS = (GB + GA - 1) / GA;                                                    \
  static_assert(GB * Q == 32, "Q must divide 32");                                             \
  static_assert(P <= 32 && P >= Q, "phase A needs Q <= P <= 32");                              \
  static_assert(NS * GA <= GB, "phase C stores NS x GA rows in a warp's GB-row buffer");

// Shared-memory tables and row buffers of one CTA (dynamic shared memory, nl_layout).
struct NLSmem {
  float4* coef;
  float2* tw;
  float* wt;
  float* sgn;
  float2* x;
  float2* y;
};

// Carve the CTA's shared memory and load the tables (the first tile's barrier publishes them).
template <int Q, int P, int NS>
__device__ __forceinline__ NLSmem nl_smem_setup(const NLArgs& a) {
  NL_CONSTS
  (void)NPASS;
  (void)RQ;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nthreads = blockDim.x;
  const NLLayout Lo = nl_layout(Q, P, a.J, a.kstride, a.rows, nthreads >> 5, GB, NS);
  NLSmem S;
  S.coef = reinterpret_cast<float4*>(smem + Lo.coef);
  S.tw = reinterpret_cast<float2*>(smem + Lo.tw);
  S.wt = reinterpret_cast<float*>(smem + Lo.wt);
  S.sgn = reinterpret_cast<float*>(smem + Lo.sgn);
  S.x = reinterpret_cast<float2*>(smem + Lo.x);
  S.y = reinterpret_cast<float2*>(smem + Lo.y);
  for (int i = threadIdx.x; i < Q * a.kstride; i += nthreads) S.coef[i] = a.coef[i];
  for (int i = threadIdx.x; i < Q * P; i += nthreads) S.tw[i] = a.tw[i];
  for (int i = threadIdx.x; i < Q * a.J; i += nthreads) {
    S.wt[i] = a.wt[i];
    S.sgn[i] = EVENP ? a.sgn[i] : 0.f;
  }
  return S;
}

// One tile (a.rows image rows of one slice, every coil and set) of the fused operator.
template <int Q, int P, int JMAX, int MODE, int NS>
__device__ __forceinline__ void nl_tile(const NLArgs& a, const NLSmem& S, int tile) {
  NL_CONSTS
  const int nthreads = blockDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = nthreads >> 5;
  float4* s_coef = S.coef;
  float2* s_tw = S.tw;
  float* s_wt = S.wt;
  float* s_sgn = S.sgn;
  float2* s_x = S.x;
  float2* s_y = S.y;
  const int J = a.J;
  const int b = tile / a.tiles_per_slice;
  const int h0 = (tile - b * a.tiles_per_slice) * a.rows;
  const int nrows = min(a.rows, a.H - h0);
  const float lam = a.lam_dev ? (float)a.lam_dev[a.lam_shared ? 0 : b] : a.lam_host;

  // ---- stage the input rows of every set (CG: p = r + beta p_old, written back)
#pragma unroll
  for (int st = 0; st < (MODE == NM_ADJ ? 0 : NS); ++st) {
    const size_t img0 = (((size_t)b * NS + st) * a.H + h0) * W;
    const int n4 = nrows * W / 2;
    const float4* src = reinterpret_cast<const float4*>(a.x + img0);
    float4* sx4 = reinterpret_cast<float4*>(s_x + st * a.rows * W);
    if (MODE == NM_CG2) {
      float4* rv = reinterpret_cast<float4*>(const_cast<float2*>(a.x) + img0);
      if (a.upd) {
        // the solve kernel's CTA holds the scalars of its one slice (FP32)
        const float be = a.first ? 0.f : a.ab_f[1];
        const float al = a.ab_f[0];
        float4* pv = reinterpret_cast<float4*>(a.pout + img0);
        float4* sv = reinterpret_cast<float4*>(a.sv + img0);
        float4* xv = reinterpret_cast<float4*>(a.xs + img0);
        const float4* wv = reinterpret_cast<const float4*>(a.out + img0);
        for (int i = threadIdx.x; i < n4; i += nthreads) {
          float4 r = rv[i], w = wv[i], x = xv[i];
          float4 pp = r, ss = w;
          if (!a.first) {
            const float4 po = pv[i], so = sv[i];
            pp.x = fmaf(be, po.x, r.x); pp.y = fmaf(be, po.y, r.y); pp.z = fmaf(be, po.z, r.z); pp.w = fmaf(be, po.w, r.w);
            ss.x = fmaf(be, so.x, w.x); ss.y = fmaf(be, so.y, w.y); ss.z = fmaf(be, so.z, w.z); ss.w = fmaf(be, so.w, w.w);
          }
          x.x = fmaf(al, pp.x, x.x); x.y = fmaf(al, pp.y, x.y); x.z = fmaf(al, pp.z, x.z); x.w = fmaf(al, pp.w, x.w);
          r.x = fmaf(-al, ss.x, r.x); r.y = fmaf(-al, ss.y, r.y); r.z = fmaf(-al, ss.z, r.z); r.w = fmaf(-al, ss.w, r.w);
          pv[i] = pp;
          sv[i] = ss;
          xv[i] = x;
          rv[i] = r;
          sx4[i] = r;
        }
      } else if (a.rhs0) {
        const float4* r0 = reinterpret_cast<const float4*>(a.rhs0 + img0);
        const float4* r0b = a.rhs0b ? reinterpret_cast<const float4*>(a.rhs0b + img0) : nullptr;
        float4* xv = reinterpret_cast<float4*>(a.xs + img0);
        for (int i = threadIdx.x; i < n4; i += nthreads) {
          float4 v = r0[i];
          if (r0b) {
            const float4 z = r0b[i];
            v = make_float4(fmaf(lam, z.x, v.x), fmaf(lam, z.y, v.y), fmaf(lam, z.z, v.z), fmaf(lam, z.w, v.w));
          }
          rv[i] = v;
          xv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
          sx4[i] = v;
        }
      } else {
        for (int i = threadIdx.x; i < n4; i += nthreads) sx4[i] = rv[i];
      }
    } else if (MODE == NM_CG) {
      const float be = a.pold ? (float)a.beta[b] : 0.f;
      const float4* po = a.pold ? reinterpret_cast<const float4*>(a.pold + img0) : nullptr;
      float4* pn = reinterpret_cast<float4*>(a.pout + img0);
      for (int i = threadIdx.x; i < n4; i += nthreads) {
        float4 v = src[i];
        if (po) {
          const float4 o = po[i];
          v.x = fmaf(be, o.x, v.x); v.y = fmaf(be, o.y, v.y);
          v.z = fmaf(be, o.z, v.z); v.w = fmaf(be, o.w, v.w);
        }
        pn[i] = v;
        sx4[i] = v;
      }
    } else {
      for (int i = threadIdx.x; i < n4; i += nthreads) sx4[i] = src[i];
    }
  }
  __syncthreads();

  const int wrow = warp / a.nwr, cgp = warp - wrow * a.nwr;
  float2* ybuf = s_y + warp * (GB * W);
  if (wrow < nrows) {
    const int h = h0 + wrow;
    const float2* xrow = s_x + wrow * W;  // set st: + st * rows * W
    const float2* map0 = a.maps + ((size_t)b * NS * a.C * a.H + h) * W;
    const size_t cstride = (size_t)a.H * W, sstride = (size_t)a.C * a.H * W;

    // ---- phase A: expand, Q-point DFT, twiddle
#pragma unroll
    for (int pass = 0; pass < (MODE == NM_ADJ ? 0 : NPASS); ++pass) {
      const int ga = lane / P, t = lane - ga * P;
      const int gi = pass * GA + ga;
      const int c = cgp * GB + gi;
      if (ga < GA && gi < GB) {
        float2 v[Q];
        if (c < a.C) {
          const float2* srow = map0 + c * cstride;
#pragma unroll
          for (int n1 = 0; n1 < Q; ++n1) v[n1] = cmul(__ldg(srow + t + P * n1), xrow[t + P * n1]);
#pragma unroll
          for (int st = 1; st < NS; ++st)
#pragma unroll
            for (int n1 = 0; n1 < Q; ++n1)
              v[n1] = cfma(__ldg(srow + st * sstride + t + P * n1), xrow[st * a.rows * W + t + P * n1], v[n1]);
        } else {
#pragma unroll
          for (int n1 = 0; n1 < Q; ++n1) v[n1] = make_float2(0.f, 0.f);
        }
        dft_pow2<Q, false>(v);
        float2* yc = ybuf + gi * W;
        yc[t] = v[0];
#pragma unroll
        for (int k1 = 1; k1 < Q; ++k1) yc[k1 * P + t] = cmul(v[k1], s_tw[k1 * P + t]);
      }
    }
    __syncwarp();

    // ---- phase B: pruned P-point DFT at the sampled frequencies and back.
    // The conjugate pairs (t, P - t) are streamed from shared memory so that
    // only the J outputs stay in registers.
    {
      const int gi = lane / Q, k1 = lane - gi * Q;
      float2* col = ybuf + gi * W + k1 * P;
      const float4* crow = s_coef + k1 * a.kstride;
      const float* wrow_ = s_wt + k1 * J;
      const float* srow_ = s_sgn + k1 * J;
      float2 X[JMAX];
      if constexpr (MODE == NM_ADJ) {
        // the sampled frequencies k = k1 + Q k2 of this lane's coil row, (-1)^k / sqrt(W) applied
        const int c = cgp * GB + gi;
        const float2* trow = a.x + (((size_t)b * a.C + (c < a.C ? c : 0)) * a.H + h) * W;
        const int* kx = a.akx + k1 * J;
        const float* fk = a.af + k1 * J;
#pragma unroll
        for (int j = 0; j < JMAX; ++j) {
          X[j] = make_float2(0.f, 0.f);
          if (j < J && c < a.C) X[j] = cscale(__ldg(trow + kx[j]), fk[j]);
        }
      } else {
      const float2 Y0 = col[0];
      float2 Ym = make_float2(0.f, 0.f);
      if (EVENP) Ym = col[P / 2];
#pragma unroll
      for (int j = 0; j < JMAX; ++j) {
        X[j] = Y0;
        if (EVENP && j < J) {
          const float sg = srow_[j];
          X[j].x = fmaf(sg, Ym.x, X[j].x);
          X[j].y = fmaf(sg, Ym.y, X[j].y);
        }
      }
#pragma unroll
      for (int q = 0; q < RQ; ++q) {
        const int t = 2 * q + 1;
        const float2 u0 = col[t], w0 = col[P - t];
        const float2 S0 = cadd(u0, w0), D0 = csub(u0, w0);
        float2 S1 = make_float2(0.f, 0.f), D1 = S1;
        if (t + 1 <= HP) {
          const float2 u1 = col[t + 1], w1 = col[P - t - 1];
          S1 = cadd(u1, w1);
          D1 = csub(u1, w1);
        }
#pragma unroll
        for (int j = 0; j < JMAX; ++j) {
          if (j < J) {
            const float4 cs = crow[j * RQ + q];
            X[j].x = fmaf(cs.x, S0.x, fmaf(cs.y, D0.y, X[j].x));
            X[j].y = fmaf(cs.x, S0.y, fmaf(-cs.y, D0.x, X[j].y));
            if (t + 1 <= HP) {
              X[j].x = fmaf(cs.z, S1.x, fmaf(cs.w, D1.y, X[j].x));
              X[j].y = fmaf(cs.z, S1.y, fmaf(-cs.w, D1.x, X[j].y));
            }
          }
        }
      }
      }
      float2 Z0 = make_float2(0.f, 0.f), Zm = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < JMAX; ++j) {
        if (j < J) {
          if (MODE != NM_ADJ) X[j] = cscale(X[j], wrow_[j]);
          Z0 = cadd(Z0, X[j]);
          if (EVENP) {
            const float sg = srow_[j];
            Zm.x = fmaf(sg, X[j].x, Zm.x);
            Zm.y = fmaf(sg, X[j].y, Zm.y);
          }
        }
      }
      __syncwarp();  // every lane has read its column before any is overwritten
      col[0] = Z0;
      if (EVENP) col[P / 2] = Zm;
#pragma unroll
      for (int q = 0; q < RQ; ++q) {
        const int t = 2 * q + 1;
        float2 A0 = make_float2(0.f, 0.f), B0 = A0, A1 = A0, B1 = A0;
#pragma unroll
        for (int j = 0; j < JMAX; ++j) {
          if (j < J) {
            const float4 cs = crow[j * RQ + q];
            A0.x = fmaf(cs.x, X[j].x, A0.x); A0.y = fmaf(cs.x, X[j].y, A0.y);
            B0.x = fmaf(cs.y, X[j].x, B0.x); B0.y = fmaf(cs.y, X[j].y, B0.y);
            A1.x = fmaf(cs.z, X[j].x, A1.x); A1.y = fmaf(cs.z, X[j].y, A1.y);
            B1.x = fmaf(cs.w, X[j].x, B1.x); B1.y = fmaf(cs.w, X[j].y, B1.y);
          }
        }
        col[t] = make_float2(A0.x - B0.y, A0.y + B0.x);
        col[P - t] = make_float2(A0.x + B0.y, A0.y - B0.x);
        if (t + 1 <= HP) {
          col[t + 1] = make_float2(A1.x - B1.y, A1.y + B1.x);
          col[P - t - 1] = make_float2(A1.x + B1.y, A1.y - B1.x);
        }
      }
    }
    __syncwarp();

    // ---- phase C: inverse twiddle, inverse Q-point DFT, conj-map combine (one sum per set)
    float2 acc[NS][Q];
#pragma unroll
    for (int st = 0; st < NS; ++st)
#pragma unroll
      for (int n1 = 0; n1 < Q; ++n1) acc[st][n1] = make_float2(0.f, 0.f);
#pragma unroll
    for (int pass = 0; pass < NPASS; ++pass) {
      const int ga = lane / P, t = lane - ga * P;
      const int gi = pass * GA + ga;
      const int c = cgp * GB + gi;
      if (ga < GA && gi < GB && c < a.C) {
        const float2* yc = ybuf + gi * W;
        float2 z[Q];
        z[0] = yc[t];
#pragma unroll
        for (int k1 = 1; k1 < Q; ++k1) z[k1] = cmulc(s_tw[k1 * P + t], yc[k1 * P + t]);
        dft_pow2<Q, true>(z);
        const float2* srow = map0 + c * cstride;
#pragma unroll
        for (int st = 0; st < NS; ++st)
#pragma unroll
          for (int n1 = 0; n1 < Q; ++n1)
            acc[st][n1] = cfmac(__ldg(srow + st * sstride + t + P * n1), z[n1], acc[st][n1]);
      }
    }
    __syncwarp();
    if (lane < GA * P) {
      const int ga = lane / P, t = lane - ga * P;
#pragma unroll
      for (int st = 0; st < NS; ++st)
#pragma unroll
        for (int n1 = 0; n1 < Q; ++n1) ybuf[(st * GA + ga) * W + t + P * n1] = acc[st][n1];
    }
  }
  __syncthreads();

  // ---- epilogue, per set: sum coil groups in fixed order, + lambda x, row partial.  The nwr
  // warps of a row split its columns (warp cgp: columns cgp * 32 + lane, stride 32 nwr); each
  // warp's share of the row partial (compensated float-float warp sum of its FP32 lane sums)
  // goes to shared memory and the shares of a row are added in warp order after the barrier.
  // The one-launch CG (NM_CG2) keeps its row partials as float-float pairs (stored in the
  // 8-byte slots of its partial arrays); the other modes store them as FP64.
  // nwarps = rows x nwr <= 8.
  __shared__ float2 s_rp[2][NS][8];
  if (wrow < nrows) {
    const int rr = wrow, h = h0 + rr;
#pragma unroll
    for (int st = 0; st < NS; ++st) {
      const size_t orow0 = (((size_t)b * NS + st) * a.H + h) * W;
      float part = 0.f, part_rr = 0.f;
      const float2* xr = s_x + (st * a.rows + rr) * W;
      const float2* rh = (MODE == NM_RESID) ? a.rhs + orow0 : nullptr;
      float2* orow = a.out + orow0;
      for (int n = cgp * 32 + lane; n < W; n += 32 * a.nwr) {
        float2 s = make_float2(0.f, 0.f);
        for (int g = 0; g < a.nwr; ++g) {
          const float2* yb = s_y + (rr * a.nwr + g) * (GB * W) + st * GA * W;
#pragma unroll
          for (int ga = 0; ga < GA; ++ga) s = cadd(s, yb[ga * W + n]);
        }
        if (MODE == NM_ADJ) {
          orow[n] = s;
          continue;
        }
        const float2 xv = xr[n];
        float2 o = make_float2(fmaf(lam, xv.x, s.x), fmaf(lam, xv.y, s.y));
        if (MODE == NM_RESID) {
          o = csub(rh[n], o);
          part = fmaf(o.x, o.x, fmaf(o.y, o.y, part));
        } else {
          part = fmaf(xv.x, o.x, fmaf(xv.y, o.y, part));
          if (MODE == NM_CG2) part_rr = fmaf(xv.x, xv.x, fmaf(xv.y, xv.y, part_rr));
        }
        orow[n] = o;
      }
      if (MODE != NM_ADJ) {
        const float2 d = warp_sum_ff(part);
        if (lane == 0) s_rp[0][st][warp] = d;
      }
      if (MODE == NM_CG2) {
        const float2 d = warp_sum_ff(part_rr);
        if (lane == 0) s_rp[1][st][warp] = d;
      }
    }
  }
  __syncthreads();
  if (MODE != NM_ADJ && a.part && (int)threadIdx.x < NS * nrows) {
    const int st = threadIdx.x / nrows, rr = threadIdx.x - st * nrows;
    const size_t prow = (size_t)b * a.HS + st * a.H + h0 + rr;
    float2 d = s_rp[0][st][rr * a.nwr], d2 = s_rp[1][st][rr * a.nwr];
    for (int g = 1; g < a.nwr; ++g) {
      d = ff_add(d, s_rp[0][st][rr * a.nwr + g]);
      if (MODE == NM_CG2) d2 = ff_add(d2, s_rp[1][st][rr * a.nwr + g]);
    }
    if (MODE == NM_CG2) {
      reinterpret_cast<float2*>(a.part)[prow] = d;
      reinterpret_cast<float2*>(a.part2)[prow] = d2;
    } else {
      a.part[prow] = ff_to_d(d);
    }
  }
}

// NS = map sets (soft-SENSE): x, out [B][NS][H][W], maps [B][NS][C][H][W]; coil image
// sum_s S_{s,c} x_s in phase A, one conj(S_{s,c}) accumulation per set in phase C.
template <int Q, int P, int JMAX, int MODE, int NS>
__global__ void __launch_bounds__(256, NS == 1 ? 3 : 2) k_normal_lines(const NLArgs a) {
  const NLSmem S = nl_smem_setup<Q, P, NS>(a);
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) nl_tile<Q, P, JMAX, MODE, NS>(a, S, tile);
  if (a.finalize) last_block(a);
}

// ------------------------------------------------------- whole CG solve in one launch
// Cooperative persistent kernel running every iteration of CG on S = A^H A + lambda I with one
// global reduction per iteration: the Chronopoulos-Gear form of the recurrence, which produces
// the iterates of the textbook (Hestenes-Stiefel) CG in exact arithmetic.  It keeps w = S r and
// s = S p (s_k = w_k + beta_{k-1} s_{k-1}) and obtains Re<p_k, S p_k> from the two inner
// products of one pass, gamma_k = ||r_k||^2 and delta_k = Re<r_k, w_k>:
//   beta_{k-1} = gamma_k / gamma_{k-1},  alpha_k = gamma_k / (delta_k - beta_{k-1} gamma_k / alpha_{k-1})
// (alpha_0 = gamma_0 / delta_0), using the orthogonality of the residuals.  Pass k (k < iters):
// staging p, s, x, r of iteration k - 1 (k >= 1), w = S r through the fused operator, row
// partials of delta and gamma, barrier of the slice.  A last pass makes the update of iteration
// iters - 1 and gamma for the residual history.  Each CTA keeps the same row tiles throughout,
// so only the row partials and the per-slice scalars cross CTAs.
//
// Barriers: the CTAs form one group per slice, and each group has an arrival count that only
// grows within the launch (barrier n completes at (n + 1) x group-size arrivals) and two release
// words.  The CTA that arrives last reduces the slice's row partials in fixed order, keeps gamma
// and alpha (FP64) for the next pass, and releases the others with the two words, which carry
// the generation and the FP32 alpha and beta the vector updates use.  One CTA reads the partials instead of every CTA reading
// them at once, and the slices do not wait for each other.  The launch is cooperative (all CTAs
// resident) and every wait is bounded: a CTA that gives up sets SENSE_STATUS_DEVICE_TIMEOUT and
// returns.
constexpr int kCoopMaxB = 16;  // slices per solve on this path

struct CgCoop {
  int iters;
  float2* x;        // solution, updated in place
  float2* r;        // residual (initial residual on entry)
  float2* p;
  float2* s;        // S p
  float2* w;        // S r
  double* hist;     // [iters + 1][B] squared residual norms or NULL
  const float2* rhs0;  // not NULL: start from x = 0, r = rhs0 (first pass)
  const float2* rhs0b;  // with rhs0, not NULL: r = rhs0 + lambda rhs0b
  float2* xlam;         // not NULL: the last pass also writes lambda x here
  // per slice b: arrival count cnt_s[32 b] and two 64-bit release words at rel_s + 32 b
  // (128-byte lines of their own), zero at launch (zeroed by the previous solve, or at workspace
  // setup)
  unsigned* cnt_s;
  unsigned* rel_s;
  // the other set of barrier words (4 KB from cnt_o), used by the previous solve: zeroed by this
  // solve after its wait for the previous kernel, for the next solve
  unsigned* cnt_o;
  double* sc;       // FP64 scalars kept for the next pass: alpha [kCoopMaxB], gamma alpha [kCoopMaxB], gamma [kCoopMaxB]
  // row partials of delta and gamma, two buffers each, used by alternate passes
  double* pd[2];
  double* pg[2];
  unsigned polls;    // release-word polls before a waiting CTA gives up
  unsigned phantom;  // arrivals each barrier expects beyond its CTAs (0; 1 only to test the timeout)
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Arrival: release of this CTA's writes (ordered before it by the CTA barrier) and acquire of
// every earlier arrival's, in one read-modify-write.
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Scalars of pass k from the row partials (delta in part, gamma in part2) of slice b, formed by
// the one CTA that completed barrier k.  gamma_{k-1} and alpha_{k-1} come from the previous
// publication.  A slice whose gamma is zero (or whose previous alpha is zero) is frozen:
// alpha = beta = 0.  With only_gamma the pass made the last update: gamma is recorded, no new
// alpha.  The row partials are float-float pairs; the sums over the rows run in float-float
// arithmetic (gamma on warp 0, delta on warp 1, side by side) and are converted to FP64 once.
// With c = gamma_{k-1} alpha_{k-1},
//   alpha_k = g / (d - beta_{k-1} g / alpha_{k-1}) = g c / (d c - g^2),  beta_{k-1} = g / gamma_{k-1},
// so one FP64 division lies on the path to alpha (warp 0) and beta's runs beside it (warp 1).
// On return (thread 0) ab[0], ab[1] hold alpha and beta in FP32 for the vector updates.
__device__ __forceinline__ void coop_scalars(const NLArgs& a, const CgCoop& c, int k, bool only_gamma,
                                             int b, float* ab, double* s_gd) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wd = (blockDim.x >> 5) > 1 ? 1 : 0;  // the warp that sums delta and divides for beta
  // gamma_{k-1}, alpha_{k-1} and their product, loaded beside the partials
  const double gp = __ldcg(c.sc + 2 * kCoopMaxB + b), ap = __ldcg(c.sc + b), gap = __ldcg(c.sc + kCoopMaxB + b);
  if (warp == 0) {
    const float2 g = warp_sum_ff(lane_tree_sum_ff(reinterpret_cast<const float2*>(a.part2) + (size_t)b * a.HS, a.HS, lane));
    if (lane == 0) s_gd[0] = ff_to_d(g);
  }
  if (warp == wd) {
    const float2 d = only_gamma ? make_float2(0.f, 0.f)
                                : warp_sum_ff(lane_tree_sum_ff(reinterpret_cast<const float2*>(a.part) + (size_t)b * a.HS, a.HS, lane));
    if (lane == 0) s_gd[1] = ff_to_d(d);
  }
  __syncthreads();
  const double g = s_gd[0], d = s_gd[1];
  const bool fin = isfinite(g) && isfinite(d);
  const bool live = fin && g > 0.0 && (k == 0 || (gp > 0.0 && ap != 0.0));
  if (lane == 0 && warp == wd && live && k > 0) s_gd[2] = g / gp;
  double al = 0.0;
  bool brk = false;
  if (threadIdx.x == 0 && live && !only_gamma) {
    const double cp = k == 0 ? 1.0 : gap;
    const double den = k == 0 ? d : d * cp - g * g;
    if (den > 0.0) al = k == 0 ? g / den : (g * cp) / den;
    else brk = true;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double be = (live && k > 0) ? s_gd[2] : 0.0;
  ab[0] = (float)al;
  ab[1] = (float)be;
  s_gd[0] = g;  // for coop_keep, after the release
  s_gd[1] = al;
  if (!fin) set_status(a.status, SENSE_DEVST_NONFINITE);
  if (brk) set_status(a.status, SENSE_DEVST_CG_BREAKDOWN);
}
// The FP64 gamma, alpha and their product of slice b for the next pass, and gamma and alpha for
// the host (thread 0 of the CTA that formed them, after the release: the next pass's last CTA
// reads them after its arrival, which the arrival chain orders after these stores).
__device__ __forceinline__ void coop_keep(const NLArgs& a, const CgCoop& c, double* hist, int b, const double* gd) {
  const double g = gd[0], al = gd[1];
  c.sc[b] = al;
  c.sc[kCoopMaxB + b] = g * al;
  c.sc[2 * kCoopMaxB + b] = g;
  a.rr[b] = g;
  a.alpha[b] = al;
  if (hist) hist[b] = g;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// A release word: the barrier generation in the high half, an FP32 scalar in the low half.
__device__ __forceinline__ unsigned long long rel_word(unsigned gen, float v) {
  return ((unsigned long long)gen << 32) | (unsigned long long)__float_as_uint(v);
}

// Barrier n of the solve with the scalars of pass k formed in between; on return ab[0], ab[1]
// (shared memory) hold the published FP32 alpha and beta of slice b0.  False if this CTA's wait
// timed out.  cnt / group: the barrier's arrival count and number of CTAs; rel: the slice's two
// 64-bit release words, each carrying generation n + 1 and one of the scalars, so a waiting CTA
// has the scalars when it sees the release.  The words are written and read with relaxed 64-bit
// accesses (no fence on the path): each word is read whole, so its scalar is that of the
// generation it carries, and no other data crosses CTAs here.  The vectors are per CTA; the row
// partials a pass writes go to the buffer of two passes back, whose reads by that pass's last
// CTA precede its next arrival, and each arrival is a release, the last one an acquire.
__device__ __forceinline__ bool coop_step(const NLArgs& a, const CgCoop& c, unsigned* cnt,
                                          unsigned long long* rel, unsigned group, int b0, unsigned n, int k,
                                          bool only_gamma, double* hist, float* ab) {
  __shared__ int s_last, s_ok;
  __shared__ double s_gd[3];
  __syncthreads();  // this CTA's partials are written
  if (threadIdx.x == 0) {
    const unsigned t = atom_add_acq_rel_u32(cnt, 1u);
    s_last = t == (n + 1u) * (group + c.phantom) - 1u;
    s_ok = 1;
  }
  __syncthreads();
  if (s_last) {
    coop_scalars(a, c, k, only_gamma, b0, ab, s_gd);
    if (threadIdx.x == 0) {
      st_relaxed_u64(rel, rel_word(n + 1u, ab[0]));
      st_relaxed_u64(rel + 1, rel_word(n + 1u, ab[1]));
      coop_keep(a, c, hist, b0, s_gd);
    }
  } else if (threadIdx.x == 0) {
    unsigned it = 0;
    for (;;) {
      const unsigned long long w0 = ld_relaxed_u64(rel), w1 = ld_relaxed_u64(rel + 1);
      if ((unsigned)(w0 >> 32) >= n + 1u && (unsigned)(w1 >> 32) >= n + 1u) {
        ab[0] = __uint_as_float((unsigned)w0);
        ab[1] = __uint_as_float((unsigned)w1);
        break;
      }
      if (++it > c.polls) {
        s_ok = 0;
        break;
      }
      __nanosleep(32);
    }
  }
  __syncthreads();
  return s_ok != 0;
}

template <int Q, int P, int JMAX, int NS>
__global__ void __launch_bounds__(256, NS == 1 ? 3 : 2) k_cg_lines(const NLArgs a0, const CgCoop c) {
  constexpr int W = Q * P;
  __shared__ float s_ab[2];  // alpha and beta of this CTA's slice (FP32, as the vector updates use them)
  const NLSmem S = nl_smem_setup<Q, P, NS>(a0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) s_ab[0] = s_ab[1] = 0.f;
  // Launched with programmatic serialisation where the driver allows it: the tables above are
  // plan constants; the vectors, partials and barrier words come after the wait.
  griddep_wait();
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) c.cnt_o[i] = 0u;
  __syncthreads();
  NLArgs a = a0;
  a.x = c.r; a.out = c.w; a.pout = c.p; a.sv = c.s; a.xs = c.x; a.ab_f = s_ab;
  a.finalize = 0;
  // One group of CTAs per slice: CTAs (b grid) / B .. ((b + 1) grid) / B - 1 take the row tiles
  // of slice b round robin, and each group has its own barrier, so the CTAs of a slice wait only
  // for each other, the slices drift apart and their phases overlap on the SMs.
  int b0 = 0;
  while (b0 + 1 < a.B && (int)(((long long)(b0 + 1) * gridDim.x) / a.B) <= (int)blockIdx.x) ++b0;
  const int g0 = (int)(((long long)b0 * gridDim.x) / a.B), g1 = (int)(((long long)(b0 + 1) * gridDim.x) / a.B);
  const int li = (int)blockIdx.x - g0;
  if (li >= a.tiles_per_slice) return;  // more CTAs than tiles in the slice: no tile, no barrier
  const int gstride = g1 - g0;
  const unsigned group = (unsigned)min(gstride, a.tiles_per_slice);
  const int b1 = b0 + 1;
  const int t0 = b0 * a.tiles_per_slice + li, t1 = b1 * a.tiles_per_slice;
  unsigned* cnt = c.cnt_s + 32 * b0;
  unsigned long long* rel = reinterpret_cast<unsigned long long*>(c.rel_s + 32 * b0);
  for (int k = 0; k < c.iters; ++k) {
    a.upd = k > 0;
    a.first = k == 1;
    a.rhs0 = k == 0 ? c.rhs0 : nullptr;
    a.rhs0b = k == 0 ? c.rhs0b : nullptr;
    a.part = (k & 1) ? c.pd[1] : c.pd[0];
    a.part2 = (k & 1) ? c.pg[1] : c.pg[0];
    for (int tile = t0; tile < t1; tile += gstride) nl_tile<Q, P, JMAX, NM_CG2, NS>(a, S, tile);
    if (!coop_step(a, c, cnt, rel, group, b0, (unsigned)k, k, false, c.hist ? c.hist + (size_t)k * a.B : nullptr,
                   s_ab)) {
      if (threadIdx.x == 0) set_status(a.status, SENSE_STATUS_DEVICE_TIMEOUT);
      return;
    }
  }
  // last update (iteration iters - 1), and the final residual with its gamma only when the
  // residual history is kept (nothing else reads them; without it the pass updates x alone and
  // ends without a barrier); one warp per row
  const bool first = c.iters == 1;
  const bool keep_r = c.hist != nullptr;
  a.part2 = (c.iters & 1) ? c.pg[1] : c.pg[0];
  for (int tile = t0; tile < t1; tile += gstride) {
    const int b = tile / a.tiles_per_slice;
    const int h0 = (tile - b * a.tiles_per_slice) * a.rows;
    const int nrows = min(a.rows, a.H - h0);
    const float al = s_ab[0], be = first ? 0.f : s_ab[1];
    const float lamx = a.lam_dev ? (float)a.lam_dev[a.lam_shared ? 0 : b] : a.lam_host;
    for (int rw = warp; rw < NS * nrows; rw += nwarps) {
      const int st = rw / nrows, h = h0 + (rw - st * nrows);
      const size_t off = ((((size_t)b * NS + st) * a.H + h) * W) / 2;
      float4* xl = c.xlam ? reinterpret_cast<float4*>(c.xlam) + off : nullptr;
      const float4* pv = reinterpret_cast<const float4*>(c.p) + off;
      const float4* sv = reinterpret_cast<const float4*>(c.s) + off;
      const float4* wv = reinterpret_cast<const float4*>(c.w) + off;
      float4* xv = reinterpret_cast<float4*>(c.x) + off;
      float4* rv = reinterpret_cast<float4*>(c.r) + off;
      float part = 0.f;
      for (int i = lane; i < W / 2; i += 32) {
        float4 r = rv[i], x = xv[i];
        float4 pp = r;
        if (!first) {
          const float4 po = pv[i];
          pp.x = fmaf(be, po.x, r.x); pp.y = fmaf(be, po.y, r.y); pp.z = fmaf(be, po.z, r.z); pp.w = fmaf(be, po.w, r.w);
        }
        x.x = fmaf(al, pp.x, x.x); x.y = fmaf(al, pp.y, x.y); x.z = fmaf(al, pp.z, x.z); x.w = fmaf(al, pp.w, x.w);
        xv[i] = x;
        if (xl) xl[i] = make_float4(lamx * x.x, lamx * x.y, lamx * x.z, lamx * x.w);
        if (keep_r) {
          const float4 w = wv[i];
          float4 ss = w;
          if (!first) {
            const float4 so = sv[i];
            ss.x = fmaf(be, so.x, w.x); ss.y = fmaf(be, so.y, w.y); ss.z = fmaf(be, so.z, w.z); ss.w = fmaf(be, so.w, w.w);
          }
          r.x = fmaf(-al, ss.x, r.x); r.y = fmaf(-al, ss.y, r.y); r.z = fmaf(-al, ss.z, r.z); r.w = fmaf(-al, ss.w, r.w);
          rv[i] = r;
          part = fmaf(r.x, r.x, fmaf(r.y, r.y, fmaf(r.z, r.z, fmaf(r.w, r.w, part))));
        }
      }
      if (keep_r) {
        const float2 d = warp_sum_ff(part);
        if (lane == 0) reinterpret_cast<float2*>(a.part2)[(size_t)b * a.HS + st * a.H + h] = d;
      }
    }
  }
  if (keep_r && !coop_step(a, c, cnt, rel, group, b0, (unsigned)c.iters, c.iters, true,
                           c.hist + (size_t)c.iters * a.B, s_ab)) {
    if (threadIdx.x == 0) set_status(a.status, SENSE_STATUS_DEVICE_TIMEOUT);
  }
}

typedef void (*CgKernel)(const NLArgs, const CgCoop);

typedef void (*NLKernel)(const NLArgs);

template <int Q, int P, int JMAX, int NS>
NLKernel pick_mode(int mode) {
  switch (mode) {
    case NM_PLAIN: return k_normal_lines<Q, P, JMAX, NM_PLAIN, NS>;
    case NM_CG: return k_normal_lines<Q, P, JMAX, NM_CG, NS>;
    case NM_RESID: return k_normal_lines<Q, P, JMAX, NM_RESID, NS>;
    default: return k_normal_lines<Q, P, JMAX, NM_ADJ, NS>;
  }
}

// Slot capacities with a compiled kernel: the smallest one >= J is used.
constexpr int kJmax[] = {4, 6, 8, 10, 12, 16};

template <int Q, int P, int NS>
CgKernel pick_cg_j(int jmax) {
  switch (jmax) {
    case 4: return k_cg_lines<Q, P, 4, NS>;
    case 6: return k_cg_lines<Q, P, 6, NS>;
    case 8: return k_cg_lines<Q, P, 8, NS>;
    case 10: return k_cg_lines<Q, P, 10, NS>;
    case 12: return k_cg_lines<Q, P, 12, NS>;
    default: return k_cg_lines<Q, P, 16, NS>;
  }
}

template <int Q, int P, int NS>
NLKernel pick_j(int jmax, int mode) {
  switch (jmax) {
    case 4: return pick_mode<Q, P, 4, NS>(mode);
    case 6: return pick_mode<Q, P, 6, NS>(mode);
    case 8: return pick_mode<Q, P, 8, NS>(mode);
    case 10: return pick_mode<Q, P, 10, NS>(mode);
    case 12: return pick_mode<Q, P, 12, NS>(mode);
    default: return pick_mode<Q, P, 16, NS>(mode);
  }
}

// Defined in normal_lines_q8.cu (Q = 8) and normal_lines_q16.cu (Q = 16); NULL if not compiled
// (ns = 2 map sets only where two sets fit a warp's phase-C buffer: P >= 16 for Q = 8, P > 16 for Q = 16).
NLKernel pick_q8(int P, int jmax, int mode, int ns);
NLKernel pick_q16(int P, int jmax, int mode, int ns);
CgKernel pick_cg_q8(int P, int jmax, int ns);
CgKernel pick_cg_q16(int P, int jmax, int ns);

}  // namespace nl
