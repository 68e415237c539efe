// Mixed-radix Stockham transforms in shared memory for the non-fused parts of
// the SENSE operator: forward A = P F C, adjoint A^H (Eq. 4) and the normal
// operator for general 2-D masks.  Each 2-D transform is a row pass (length W)
// and a column pass (length H) through global memory.
//
// Centred unitary DFT along one axis of even length L:
//   F_c[k, n] = L^{-1/2} e^{-2 pi i (k - L/2)(n - L/2)/L}
//             = (-1)^{L/2} L^{-1/2} (-1)^k e^{-2 pi i k n / L} (-1)^n,
// i.e. a plain DFT between two (-1)^n modulations.  For the normal operator the
// modulations cancel against each other (F^H diag(m) F is circulant), so that
// path uses a plain DFT pair and the mask shifted to plain frequency order.
//
// Passes that hold their transforms in registers (threads own a few points each; exchanges
// through shared memory between radix stages):
//   - 512 points (8 x 8 x 8, 64 threads per sequence): the Toeplitz operator's row and column
//     passes for 2H = 512 or 2W = 512 (non-Cartesian SENSE, Sec. 2.3.3), and Bluestein's
//     512-point convolution for the normal operator's row DFTs of other widths up to 256;
//   - 256 points (8 x 8 x 4, 32 threads per column): the normal operator's column pass, H = 256;
//   - W = 8 P points (P prime 17 .. 31, one warp per row): the normal operator's row DFTs, the
//     P-point DFTs as direct sums over conjugate pairs.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "plan.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kRows = 4;   // rows per CTA in row passes
constexpr int kCols = 8;   // columns per CTA in column passes
constexpr int kMaxPer = 16;  // accumulator slots per thread: kRows * W <= kThreads * kMaxPer

struct Fft1DDev {
  int L, nst;
  int radix[SENSE_MAX_STAGES];
  const float2* tw;
};

template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2 (&v)[R], const float2* tw, int L) {
  if constexpr ((R & (R - 1)) == 0) {
    dft_pow2<R, INV>(v);
  } else {
    float2 X[R];
    const int step = L / R;
    float2 s = v[0];
#pragma unroll
    for (int t = 1; t < R; ++t) s = cadd(s, v[t]);
    X[0] = s;
#pragma unroll
    for (int k = 1; k < R; ++k) {
      float2 acc = v[0];
#pragma unroll
      for (int t = 1; t < R; ++t) {
        const float2 w = __ldg(tw + step * ((t * k) % R));
        acc = INV ? cfmac(w, v[t], acc) : cfma(v[t], w, acc);
      }
      X[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = X[k];
  }
}

// One radix-R Stockham butterfly j of a stage whose sub-transforms have length Ns.
template <int R, bool INV>
__device__ __forceinline__ void bfly(const float2* in, float2* out, int j, int Ns, int L,
                                     const float2* tw) {
  const int stride = L / R;
  float2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = in[j + r * stride];
  const int k = j % Ns;
  if (Ns > 1) {
    // one table load per butterfly; w^r = w^(r-1) w (rounding stays within a few ulp for R <= 8)
    const float2 w1 = __ldg(tw + k * (L / (Ns * R)));
    float2 w = w1;
#pragma unroll
    for (int r = 1; r < R; ++r) {
      if (r > 1) w = cmul(w, w1);
      v[r] = INV ? cmulc(w, v[r]) : cmul(v[r], w);
    }
  }
  dft_small<R, INV>(v, tw, L);
  const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) out[idxD + r * Ns] = v[r];
}

// Radix-R stage for the larger primes with the stage twiddles already applied to the inputs
// (y_r = in[j + r L/R] w^{r (j mod Ns) L/(Ns R)}): the R-point DFT over r for the output pair
// (p, R - p) of work item j.  Inputs r and R - r enter as S_r = y_r + y_{R-r} and
// D_r = y_r - y_{R-r}:  X_p = A -/+ i B,  X_{R-p} = A +/- i B  (forward / inverse) with
// A = y_0 + sum_r cos(2 pi r p / R) S_r and B = sum_r sin(2 pi r p / R) D_r, r = 1 .. (R - 1)/2,
// so each pair of outputs costs (R - 1)/2 table loads and 2 (R - 1) multiply-adds.  p = 0 gives
// X_0 = sum_r y_r.
template <bool INV>
__device__ __forceinline__ void bfly_pair(const float2* in, float2* out, int j, int p, int R, int Ns, int L,
                                          const float2* tw) {
  const int stride = L / R, jm = j % Ns;
  const int o0 = (j / Ns) * Ns * R + jm;  // output k goes to o0 + k Ns
  const float2 y0 = in[j];
  if (p == 0) {
    float2 sum = y0;
    for (int r = 1; r < R; ++r) sum = cadd(sum, in[j + r * stride]);
    out[o0] = sum;
    return;
  }
  float2 A = y0, Bs = make_float2(0.f, 0.f);
  const int step = p * stride;  // angle index of r = 1 in the length-L table
  int idx = 0;
  for (int r = 1; r <= (R - 1) / 2; ++r) {
    idx += step;
    if (idx >= L) idx -= L;
    const float2 w = __ldg(tw + idx);  // (cos t, -sin t), t = 2 pi r p / R
    const float2 u = in[j + r * stride], v = in[j + (R - r) * stride];
    const float2 S = cadd(u, v), D = csub(u, v);
    A.x = fmaf(w.x, S.x, A.x);
    A.y = fmaf(w.x, S.y, A.y);
    Bs.x = fmaf(-w.y, D.x, Bs.x);
    Bs.y = fmaf(-w.y, D.y, Bs.y);
  }
  const float2 mib = make_float2(Bs.y, -Bs.x);  // -i B
  const float2 plus = cadd(A, mib), minus = csub(A, mib);
  out[o0 + p * Ns] = INV ? minus : plus;
  out[o0 + (R - p) * Ns] = INV ? plus : minus;
}

// Power-of-two lengths with the stage structure fixed at compile time: the same radix order as
// the generic plan (radix 8 while it divides, then one radix 4 or 2 stage), the same twiddles
// and butterflies, with every stride, mask and shift a constant (no per-butterfly divisions or
// radix dispatch).
// Intermediate results between two stages are stored with the index swizzled inside blocks of
// 16 (i ^ ((i >> 4) & 7)): the first stage writes each work item's R outputs R elements apart,
// which in natural order puts 16 lanes on two 8-byte bank slots; swizzled they take 16.  Reads of
// 16 consecutive elements stay conflict-free.  Input and final output are in natural order.
template <int L>
__device__ __forceinline__ int p2_swz(int i) {
  return L >= 16 ? (i ^ ((i >> 4) & 7)) : i;
}

// ZHI: the upper half of the transform's input is zero (a zero-padded sequence): in the first
// stage (NS = 1) input j + r L/R lies in the upper half exactly when r >= R/2, so those loads are
// skipped.  HOUT: only the lower half of the output is used: in the last stage (NS R = L) output
// k + r NS lies in the lower half exactly when r < R/2, so the other stores are skipped.
template <int R, bool INV, int NS, int L, bool ZHI = false, bool HOUT = false>
__device__ __forceinline__ void bfly_p2(const float2* in, float2* out, int j, const float2* tw) {
  constexpr int stride = L / R;
  constexpr bool SWZ_IN = NS > 1;       // written by an earlier stage
  constexpr bool SWZ_OUT = NS * R < L;  // read by a later stage
  constexpr bool ZERO_HI = ZHI && NS == 1;
  constexpr bool STORE_LO = HOUT && NS * R == L;
  float2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r)
    v[r] = (ZERO_HI && 2 * r >= R) ? make_float2(0.f, 0.f) : in[SWZ_IN ? p2_swz<L>(j + r * stride) : j + r * stride];
  const int k = j & (NS - 1);
  if constexpr (NS > 1) {
    // one table load per butterfly: w^r for r >= 2 as products of w (at most three deep), so the
    // twiddle loads do not saturate the L1 pipe (rounding of w^r stays within a few ulp)
    float2 w[R];
    w[1] = __ldg(tw + k * (L / (NS * R)));
    if constexpr (R >= 4) {
      w[2] = cmul(w[1], w[1]);
      w[3] = cmul(w[2], w[1]);
    }
    if constexpr (R == 8) {
      w[4] = cmul(w[2], w[2]);
      w[5] = cmul(w[4], w[1]);
      w[6] = cmul(w[4], w[2]);
      w[7] = cmul(w[4], w[3]);
    }
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = INV ? cmulc(w[r], v[r]) : cmul(v[r], w[r]);
  }
  dft_pow2<R, INV>(v);
  const int idxD = (j / NS) * NS * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (!STORE_LO || 2 * r < R) out[SWZ_OUT ? p2_swz<L>(idxD + r * NS) : idxD + r * NS] = v[r];
}

template <bool INV, int L, int NS, bool ZHI = false, bool HOUT = false>
__device__ __forceinline__ float2* fft_p2(float2* a, float2* b, int ntr, const float2* tw, int ld) {
  if constexpr (NS >= L) {
    return a;
  } else {
    constexpr int R = (L / NS >= 8) ? 8 : L / NS;
    constexpr int NB = L / R;
    for (int w = threadIdx.x; w < ntr * NB; w += blockDim.x) {
      const int tr = w / NB, j = w - tr * NB;
      bfly_p2<R, INV, NS, L, ZHI, HOUT>(a + tr * ld, b + tr * ld, j, tw);
    }
    __syncthreads();
    return fft_p2<INV, L, NS * R, ZHI, HOUT>(b, a, ntr, tw, ld);
  }
}

// True where fft_smem_half takes a compile-time power-of-two plan (and so honours ZHI / HOUT).
template <int CLS>
__device__ __forceinline__ bool p2_plan(int L) {
  return CLS == 0 && (L == 64 || L == 128 || L == 256 || L == 512 || L == 1024);
}

// fft_smem for a zero-padded input (ZHI: the upper half of every sequence is zero and need not
// be stored) and/or a half-length result (HOUT: only the lower half is valid on return).  Lengths
// without a compile-time plan fall back to the full transform: the caller then stores the zeros
// and reads only the lower half.
template <bool INV, int CLS, bool ZHI, bool HOUT>
__device__ float2* fft_smem_half(float2* a, float2* b, int ntr, const Fft1DDev& f, int ld);

// Transform ntr sequences of length L held in a at stride ld (>= L; ping-pong with b).  Column
// passes use ld = L + 1: the transposing loads and stores of neighbouring columns then fall into
// different shared-memory banks.  Returns the buffer holding the result.  All threads take part.
// CLS selects the radices compiled into the stage loop: 0 = {2, 4, 8}, 1 = also {3, 5, 7},
// 2 = also the primes 11 .. 31 (stage twiddles applied in place, then one output pair per work
// item, bfly_pair; a is overwritten).  The radix 3 - 7 butterflies hold R complex values in
// registers; leaving them out of class 0 keeps power-of-two transforms at the lowest register
// counts.
template <bool INV, int CLS>
__device__ float2* fft_smem(float2* a, float2* b, int ntr, const Fft1DDev& f, int ld) {
  const int L = f.L;
  if constexpr (CLS == 0) {  // compile-time plans for the common power-of-two lengths
    switch (L) {
      case 64: return fft_p2<INV, 64, 1>(a, b, ntr, f.tw, ld);
      case 128: return fft_p2<INV, 128, 1>(a, b, ntr, f.tw, ld);
      case 256: return fft_p2<INV, 256, 1>(a, b, ntr, f.tw, ld);
      case 512: return fft_p2<INV, 512, 1>(a, b, ntr, f.tw, ld);
      case 1024: return fft_p2<INV, 1024, 1>(a, b, ntr, f.tw, ld);
      default: break;
    }
  }
  int Ns = 1;
  for (int s = 0; s < f.nst; ++s) {
    const int R = f.radix[s];
    const int nb = L / R;
    if (CLS >= 2 && R >= 11) {
      // stage twiddles in place (element j + r L/R, j mod Ns = jm: w^{r jm L/(Ns R)}), then the
      // R-point DFTs one output pair per work item
      if (Ns > 1) {
        const int tws = L / (Ns * R);
        for (int w = threadIdx.x; w < ntr * L; w += blockDim.x) {
          const int tr = w / L, i = w - tr * L;
          const int r = i / nb, jm = (i - r * nb) % Ns;
          if (r > 0 && jm > 0) {
            float2* e = a + tr * ld + i;
            const float2 t = __ldg(f.tw + r * jm * tws);
            *e = INV ? cmulc(t, *e) : cmul(*e, t);
          }
        }
        __syncthreads();
      }
      const int np = (R + 1) / 2;  // p = 0 .. (R - 1)/2
      for (int w = threadIdx.x; w < ntr * nb * np; w += blockDim.x) {
        const int tr = w / (nb * np), rem = w - tr * nb * np;
        const int pp = rem / nb, j = rem - pp * nb;
        bfly_pair<INV>(a + tr * ld, b + tr * ld, j, pp, R, Ns, L, f.tw);
      }
      __syncthreads();
      float2* t = a; a = b; b = t;
      Ns *= R;
      continue;
    }
    for (int w = threadIdx.x; w < ntr * nb; w += blockDim.x) {
      const int tr = w / nb, j = w - tr * nb;
      const float2* in = a + tr * ld;
      float2* out = b + tr * ld;
      switch (R) {
        case 2: bfly<2, INV>(in, out, j, Ns, L, f.tw); break;
        case 4: bfly<4, INV>(in, out, j, Ns, L, f.tw); break;
        case 8: bfly<8, INV>(in, out, j, Ns, L, f.tw); break;
        default:
          if constexpr (CLS >= 1) {
            switch (R) {
              case 3: bfly<3, INV>(in, out, j, Ns, L, f.tw); break;
              case 5: bfly<5, INV>(in, out, j, Ns, L, f.tw); break;
              case 7: bfly<7, INV>(in, out, j, Ns, L, f.tw); break;
              default: break;
            }
          }
      }
    }
    __syncthreads();
    float2* t = a; a = b; b = t;
    Ns *= R;
  }
  return a;
}

template <bool INV, int CLS, bool ZHI, bool HOUT>
__device__ float2* fft_smem_half(float2* a, float2* b, int ntr, const Fft1DDev& f, int ld) {
  if constexpr (CLS == 0) {
    switch (f.L) {
      case 64: return fft_p2<INV, 64, 1, ZHI, HOUT>(a, b, ntr, f.tw, ld);
      case 128: return fft_p2<INV, 128, 1, ZHI, HOUT>(a, b, ntr, f.tw, ld);
      case 256: return fft_p2<INV, 256, 1, ZHI, HOUT>(a, b, ntr, f.tw, ld);
      case 512: return fft_p2<INV, 512, 1, ZHI, HOUT>(a, b, ntr, f.tw, ld);
      case 1024: return fft_p2<INV, 1024, 1, ZHI, HOUT>(a, b, ntr, f.tw, ld);
      default: break;
    }
  }
  return fft_smem<INV, CLS>(a, b, ntr, f, ld);
}

__device__ __forceinline__ float pm1(int n) { return (n & 1) ? -1.f : 1.f; }

// Row pass, expanding by the coil maps:  T[b,c,h,:] = DFT_W(S_c x) with
//   mode 0 (forward): input (-1)^{h+w} S x, output (-1)^{kw} (-1)^{W/2} / sqrt(W)
//   mode 1 (normal):  plain DFT, no modulation, no scale.
template <int CLS>
__global__ void __launch_bounds__(kThreads, 2) k_row_expand(int B, int S, int C, int H, const float2* x,
                                                         const float2* maps, float2* T,
                                                         Fft1DDev f, int mode) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = f.L;
  float2* a = reinterpret_cast<float2*>(smem);
  float2* bb = a + kRows * W;
  const int bc = blockIdx.y, b = bc / C, c = bc - b * C;
  const int h0 = blockIdx.x * kRows;
  const int nr = min(kRows, H - h0);
  for (int i = threadIdx.x; i < nr * W; i += blockDim.x) {
    const int r = i / W, w = i - r * W, h = h0 + r;
    // coil image: sum over the map sets of S_{s,c} x_s (maps [B][S][C][H][W], x [B][S][H][W])
    float2 v = make_float2(0.f, 0.f);
    for (int s = 0; s < S; ++s)
      v = cfma(maps[((((size_t)b * S + s) * C + c) * H + h) * W + w], x[(((size_t)b * S + s) * H + h) * W + w], v);
    if (mode == 0) v = cscale(v, pm1(h + w));
    a[i] = v;
  }
  __syncthreads();
  float2* res = fft_smem<false, CLS>(a, bb, nr, f, W);
  const float sc = (mode == 0) ? pm1(W / 2) * rsqrtf((float)W) : 1.f;
  for (int i = threadIdx.x; i < nr * W; i += blockDim.x) {
    const int r = i / W, k = i - r * W;
    float2 v = res[i];
    if (mode == 0) v = cscale(v, sc * pm1(k));
    T[(((size_t)b * C + c) * H + h0 + r) * W + k] = v;
  }
}

// Column pass over data [B*C][H][W], kCols columns per CTA (src may equal dst).
//   mode 0 (forward):  dst = M (-1)^{kh} (-1)^{H/2}/sqrt(H) DFT_H(src)
//   mode 1 (adjoint):  dst = (-1)^h (-1)^{H/2}/sqrt(H) IDFT_H((-1)^{kh} M src)
//   mode 2 (normal):   dst = IDFT_H(m2s DFT_H(src))   (m2s: mask^2/(HW), plain order)
// mask: modes 0/1 the centred mask ([W] if lines else [H][W]); mode 2 shifted mask^2.
// cols (optional): transform only the ncols listed columns (mode 1 with a line mask: the sampled
// ones; the other columns of dst are left untouched).
template <int CLS>
__global__ void __launch_bounds__(kThreads, 2) k_col(int W, const float2* src, float2* dst,
                                                  Fft1DDev f, const float* mask, int lines,
                                                  int mode, const int* cols, int ncols) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int H = f.L, ld = H + 1;
  float2* a = reinterpret_cast<float2*>(smem);
  float2* bb = a + kCols * ld;
  const int bc = blockIdx.y;
  const int w0 = blockIdx.x * kCols;
  const int nc = min(kCols, (cols ? ncols : W) - w0);
  const size_t base = (size_t)bc * H * W;
  auto colw = [&](int cc) { return cols ? cols[w0 + cc] : w0 + cc; };
  for (int i = threadIdx.x; i < H * kCols; i += blockDim.x) {
    const int h = i / kCols, cc = i - h * kCols;
    float2 v = make_float2(0.f, 0.f);
    if (cc < nc) {
      v = src[base + (size_t)h * W + colw(cc)];
      if (mode == 1) {
        const int w = colw(cc);
        const float m = lines ? mask[w] : mask[(size_t)h * W + w];
        v = cscale(v, m * pm1(h));
      }
    }
    a[cc * ld + h] = v;
  }
  __syncthreads();
  float2* res;
  if (mode == 1) {
    res = fft_smem<true, CLS>(a, bb, kCols, f, ld);
  } else {
    res = fft_smem<false, CLS>(a, bb, kCols, f, ld);
    if (mode == 2) {
      float2* other = (res == a) ? bb : a;
      for (int i = threadIdx.x; i < H * kCols; i += blockDim.x) {
        const int cc = i / H, k = i - cc * H;
        const int w = colw(cc < nc ? cc : 0);
        float m = 0.f;
        if (cc < nc) m = lines ? mask[w] : mask[(size_t)k * W + w];
        res[cc * ld + k] = cscale(res[cc * ld + k], m);
      }
      __syncthreads();
      res = fft_smem<true, CLS>(res, other, kCols, f, ld);
    }
  }
  const float sc = pm1(H / 2) * rsqrtf((float)H);
  for (int i = threadIdx.x; i < H * kCols; i += blockDim.x) {
    const int h = i / kCols, cc = i - h * kCols;
    if (cc >= nc) continue;
    float2 v = res[cc * ld + h];
    const int w = colw(cc);
    if (mode == 0) {
      const float m = lines ? mask[w] : mask[(size_t)h * W + w];
      v = cscale(v, sc * pm1(h) * m);
    } else if (mode == 1) {
      v = cscale(v, sc * pm1(h));
    }
    dst[base + (size_t)h * W + w] = v;
  }
}

// 16-byte asynchronous global -> shared copies: the inverse row passes copy the next coil's rows
// into a third shared buffer while the current coil is transformed (smem_rows_inv bytes).
__device__ __forceinline__ void tp_cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void tp_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tp_cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
int smem_rows_inv(int W2) { return 3 * kRows * W2 * (int)sizeof(float2); }

// Row pass with coil combination:
//   out[b,h,:] = sum_c conj(S_c) post(IDFT_W(pre(T[b,c,h,:]))) (+ lambda xin)
//   mode 1 (adjoint): pre (-1)^{kw}, post (-1)^w (-1)^{W/2}/sqrt(W)
//   mode 2 (normal):  no modulation, no scale (the scale sits in the mask table)
// With cpg < C (one map set only), CTA z sums coils z cpg .. z cpg + cpg - 1 and writes that
// partial sum over the rows of coil z cpg it has just read (no other CTA reads them);
// k_coil_groups_sum then adds the groups in fixed order.  The next coil's rows are copied in
// while the current one is transformed.
template <int CLS>
__global__ void __launch_bounds__(kThreads, 2) k_row_combine(int S, int C, int H, float2* T,
                                                          const float2* maps, float2* out,
                                                          Fft1DDev f, int mode,
                                                          const float2* xin, float lam_host,
                                                          const double* lam_dev, int cpg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = f.L;
  float2* const base = reinterpret_cast<float2*>(smem);  // three buffers of kRows x W
  const int bstride = kRows * W;
  const int b = blockIdx.y / S, s = blockIdx.y - b * S;  // output set s of slice b
  const int h0 = blockIdx.x * kRows;
  const int nr = min(kRows, H - h0);
  const int c0 = blockIdx.z * cpg, c1 = min(C, c0 + cpg);
  const int n16 = nr * W / 2;  // 16-byte chunks of one coil's rows (W even)
  auto fetch = [&](int c, float2* dst) {
    const float2* src = T + (((size_t)b * C + c) * H + h0) * W;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) tp_cp_async16(dst + 2 * i, src + 2 * i);
    tp_cp_async_commit();
  };
  float2 acc[kMaxPer];
#pragma unroll
  for (int e = 0; e < kMaxPer; ++e) acc[e] = make_float2(0.f, 0.f);
  const float sc = pm1(W / 2) * rsqrtf((float)W);
  int ip = 0, is = 1, iq = 2;  // prefetched input, FFT scratch, next prefetch
  fetch(c0, base + ip * bstride);
  for (int c = c0; c < c1; ++c) {
    float2* a = base + ip * bstride;
    tp_cp_async_wait_all();
    __syncthreads();
    if (c + 1 < c1) fetch(c + 1, base + iq * bstride);
    if (mode == 1) {  // (-1)^k on the input (each thread its own copied chunks)
      for (int i = threadIdx.x; i < n16; i += blockDim.x)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int k = (2 * i + q) % W;
          a[2 * i + q] = cscale(a[2 * i + q], pm1(k));
        }
      __syncthreads();
    }
    float2* res = fft_smem<true, CLS>(a, base + is * bstride, nr, f, W);
#pragma unroll
    for (int e = 0; e < kMaxPer; ++e) {
      const int i = threadIdx.x + e * blockDim.x;
      if (i < nr * W) {
        const int r = i / W, w = i - r * W;
        float2 v = res[i];
        if (mode == 1) v = cscale(v, sc * pm1(w));
        const float2 sm = maps[((((size_t)b * S + s) * C + c) * H + h0 + r) * W + w];
        acc[e] = cfmac(sm, v, acc[e]);
      }
    }
    __syncthreads();
    const int t = ip;
    ip = iq;
    iq = t;
  }
  if (cpg < C) {  // partial sum of this coil group
    float2* dst = T + (((size_t)b * C + c0) * H + h0) * W;
#pragma unroll
    for (int e = 0; e < kMaxPer; ++e) {
      const int i = threadIdx.x + e * blockDim.x;
      if (i < nr * W) dst[i] = acc[e];
    }
    return;
  }
  const float lam = lam_dev ? (float)lam_dev[b] : lam_host;
#pragma unroll
  for (int e = 0; e < kMaxPer; ++e) {
    const int i = threadIdx.x + e * blockDim.x;
    if (i < nr * W) {
      const size_t o = (((size_t)b * S + s) * H + h0) * W + i;
      float2 v = acc[e];
      if (xin) {
        const float2 xv = xin[o];
        v.x = fmaf(lam, xv.x, v.x);
        v.y = fmaf(lam, xv.y, v.y);
      }
      out[o] = v;
    }
  }
}

// out[b] = sum over coil groups g (in order) of T[b, g cpg] (+ lambda xin[b]); one map set.  T
// holds H rows of ldT entries per coil, of which the first W are used.
__global__ void k_coil_groups_sum(int B, int C, int H, int W, int ldT, int cpg, const float2* T, const float2* xin,
                                  float lam_host, const double* lam_dev, float2* out) {
  const int HW = H * W;
  const size_t n = (size_t)B * HW;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / HW);
    const int q = (int)(i - (size_t)b * HW);
    const int h = q / W, w = q - h * W;
    float2 v = make_float2(0.f, 0.f);
    for (int c = 0; c < C; c += cpg) {
      const float2 t = T[(((size_t)b * C + c) * H + h) * ldT + w];
      v.x += t.x;
      v.y += t.y;
    }
    if (xin) {
      const float lam = lam_dev ? (float)lam_dev[b] : lam_host;
      const float2 xv = xin[i];
      v.x = fmaf(lam, xv.x, v.x);
      v.y = fmaf(lam, xv.y, v.y);
    }
    out[i] = v;
  }
}

// ------------------------------------------------ Toeplitz embedding (non-Cartesian)
// F^H P^H P F u = crop(IFFT2(psf_hat * FFT2(pad(u)))) on the 2H x 2W grid, with psf_hat holding
// the 1 / (4 H W) of the inverse.  Rows H .. 2H - 1 of pad(u) are zero, so only H rows are
// transformed along W, and the column pass keeps only rows 0 .. H - 1 of its result.
//   k_tp_rows_fwd:  T[b,c,h,:] = FFT_2W(S_c x [b,h,0..W-1], zero-padded)          h < H
//   k_tp_cols:      T[:,kw] (rows < H) = rows < H of IFFT_2H(psf_hat[:,kw] FFT_2H(T[:,kw] padded))
//   k_tp_rows_inv:  out[b,h,:] = sum_c conj(S_c) IFFT_2W(T[b,c,h,:])[0..W-1] + lambda x
// T is [B][C][H][2W].
template <int CLS>
__global__ void __launch_bounds__(kThreads, 2) k_tp_rows_fwd(int C, int H, int W, const float2* x,
                                                          const float2* maps, float2* T, Fft1DDev f) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W2 = f.L;
  float2* a = reinterpret_cast<float2*>(smem);
  float2* bb = a + kRows * W2;
  const int bc = blockIdx.y, b = bc / C;
  const int h0 = blockIdx.x * kRows;
  const int nr = min(kRows, H - h0);
  // the zero half of each padded row is stored only for a transform without the pruned plan
  const int wst = p2_plan<CLS>(W2) ? W : W2;
  for (int i = threadIdx.x; i < nr * wst; i += blockDim.x) {
    const int r = i / wst, w = i - r * wst, h = h0 + r;
    float2 v = make_float2(0.f, 0.f);
    if (w < W) v = cmul(maps[((size_t)bc * H + h) * W + w], x[((size_t)b * H + h) * W + w]);
    a[r * W2 + w] = v;
  }
  __syncthreads();
  float2* res = fft_smem_half<false, CLS, true, false>(a, bb, nr, f, W2);
  for (int i = threadIdx.x; i < nr * W2; i += blockDim.x)
    T[((size_t)bc * H + h0) * W2 + i] = res[i];
}

template <int CLS>
__global__ void __launch_bounds__(kThreads, 3) k_tp_cols(int H, int W2, float2* T, Fft1DDev f,
                                                      const float2* psf_hat) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int H2 = f.L, ld = H2 + 1;
  float2* a = reinterpret_cast<float2*>(smem);
  float2* bb = a + kCols * ld;
  const int bc = blockIdx.y;
  const int w0 = blockIdx.x * kCols;
  const int nc = min(kCols, W2 - w0);
  const size_t base = (size_t)bc * H * W2;
  const int hst = p2_plan<CLS>(H2) ? H : H2;  // rows H .. 2H - 1 are zero (stored only without the pruned plan)
  for (int i = threadIdx.x; i < hst * kCols; i += blockDim.x) {
    const int h = i / kCols, cc = i - h * kCols;
    float2 v = make_float2(0.f, 0.f);
    if (cc < nc && h < H) v = T[base + (size_t)h * W2 + w0 + cc];
    a[cc * ld + h] = v;
  }
  __syncthreads();
  float2* res = fft_smem_half<false, CLS, true, false>(a, bb, kCols, f, ld);
  float2* other = (res == a) ? bb : a;
  for (int i = threadIdx.x; i < H2 * kCols; i += blockDim.x) {
    const int h = i / kCols, cc = i - h * kCols;  // psf_hat read along its rows
    const float2 ph = cc < nc ? psf_hat[(size_t)h * W2 + w0 + cc] : make_float2(0.f, 0.f);
    res[cc * ld + h] = cmul(res[cc * ld + h], ph);
  }
  __syncthreads();
  res = fft_smem_half<true, CLS, false, true>(res, other, kCols, f, ld);  // rows < H only
  for (int i = threadIdx.x; i < H * kCols; i += blockDim.x) {
    const int h = i / kCols, cc = i - h * kCols;
    if (cc < nc) T[base + (size_t)h * W2 + w0 + cc] = res[cc * ld + h];
  }
}

// ---------------------------------------- 512-point transforms held in registers
// The Toeplitz passes along a length-512 axis (2H = 512 for the column pass, 2W = 512 for the
// row passes) keep each sequence in the registers of 64 threads, 8 points each: 512 = 8 x 8 x 8,
// three radix-8 stages with two exchanges through shared memory per transform (the generic
// passes move every element through shared memory once per stage and twice more for the
// transposing load and store).  Index digits, base 8, of one sequence (all sums over one digit
// are 8-point DFTs in registers; w = e^{-2 pi i / 512}; thread t = lo + 8 hi of the sequence):
//   forward, input n = 64 n1 + n2 (n1 < 4: the upper half is the zero padding):
//     s1  t = n2:            Y[n2][k1]  = w^{n2 k1} sum_{n1} x[64 n1 + n2] w^{64 n1 k1}
//     s2  t = m2 + 8 k1:     V[k1][m2][j1] = w^{8 m2 j1} sum_{m1} Y[8 m1 + m2][k1] w^{64 m1 j1}
//     s3  t = j1 + 8 k1:     X[k1 + 8 j1 + 64 j2] = sum_{m2} V[k1][m2][j1] w^{64 m2 j2}
//   inverse, in decimation-in-frequency order from the layout s3 leaves (k = d0 + 8 d1 + 64 d2,
//   output n = e0 + 8 e1 + 64 e2; only e2 < 4, the first half, is formed):
//     A   t = d1 + 8 d0:     U[d0][d1][e0] = w^{-8 d1 e0} sum_{d2} P[k] w^{-64 d2 e0}
//     B   t = e0 + 8 d0:     Z[d0][e0][e1] = w^{-d0 (e0 + 8 e1)} sum_{d1} U[d0][d1][e0] w^{-64 d1 e1}
//     C   t = e0 + 8 e1:     y[e0 + 8 e1 + 64 e2] = sum_{d0} Z[d0][e0][e1] w^{-64 d0 e2}
// Shared layouts of Y, V (and U), Z per sequence: with the column pass's lanes (8 columns x 4
// threads per warp, sequence stride 514 = 2 mod 16 float2) Y at 64 k1 + n2, V at
// 64 a + 8 b + ((c + b) & 7) for [a][b][c], Z at e0 + 8 e1 + 64 d0; with the row passes' lanes
// (32 threads of one row) the same with the rotations and flips that put the two values of hi
// in a half-warp on different bank halves.  Either way the 16 lanes of every half-warp access 16
// different bank pairs on every exchange.
template <bool ROW>
struct Lay512 {
  static __device__ __forceinline__ int y(int n2, int k1) { return 64 * k1 + (ROW ? ((n2 + 8 * k1) & 63) : n2); }
  static __device__ __forceinline__ int v(int a, int b, int c) {
    return 64 * a + 8 * (ROW ? (b ^ (a & 1)) : b) + ((c + b) & 7);
  }
  static __device__ __forceinline__ int z(int d0, int e0, int e1) {
    return e0 + 8 * (ROW ? (e1 ^ (d0 & 1)) : e1) + 64 * d0;
  }
};

// 8-point DFT of (x0, x1, x2, x3, 0, 0, 0, 0): even outputs the 4-point DFT of x, odd outputs
// the 4-point DFT of x_n e^{-/+ 2 pi i n / 8}.
template <bool INV>
__device__ __forceinline__ void dft8_lowhalf(float2 (&v)[8]) {
  float2 e[4] = {v[0], v[1], v[2], v[3]};
  float2 o[4] = {v[0], cmul_tw<INV>(v[1], 1, 8), cmul_tw<INV>(v[2], 2, 8), cmul_tw<INV>(v[3], 3, 8)};
  dft_pow2<4, INV>(e);
  dft_pow2<4, INV>(o);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = e[k];
    v[2 * k + 1] = o[k];
  }
}

// Twiddles of the thread with index t = lo + 8 hi of its sequence, the same for every sequence:
// slots 1 .. 7 w^{t j} (s1), 9 .. 15 w^{8 lo j} (s2 and, conjugated, A), 16 .. 23
// w^{hi (lo + 8 e1)} (B); slots 0 and 8 hold 1.  The plan holds the kTw512 x 64 table,
// slot-major (lanes with consecutive t read consecutive entries, the threads of sequences that
// share t the same entry); a CTA copies it into shared memory once (tw_copy, then a barrier).
constexpr int kTw512 = 24;
constexpr int kTwTab = 64 * kTw512;  // float2 per table
// exponent of slot s of thread t, in units of 2 pi / 512
SENSE_HD int tw512_exp(int s, int t) {
  const int lo = t & 7, hi = t >> 3;
  return (s < 8 ? t * s : (s < 16 ? 8 * lo * (s - 8) : hi * (lo + 8 * (s - 16)))) & 511;
}
// n float2 (n even, both addresses 16-byte aligned), all threads of the CTA
__device__ __forceinline__ void tw_copy(float2* tab, const float2* __restrict__ g, int n) {
  const float4* src = reinterpret_cast<const float4*>(g);
  float4* dst = reinterpret_cast<float4*>(tab);
  for (int i = threadIdx.x; i < n / 2; i += blockDim.x) dst[i] = __ldg(src + i);
}
// dst[addr(j)] = v[j] * w_j (CONJ: conj(w_j) * v[j]) with w_j table slot o + j of the thread
// (tabt = tab + t), j = 0 .. 7, slot o skipped where it holds 1 (ONE0).
template <bool CONJ, bool ONE0, typename Addr>
__device__ __forceinline__ void tw512_apply(float2 (&v)[8], const float2* tabt, int o, float2* dst, Addr addr) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (ONE0 && j == 0) {
      dst[addr(0)] = v[0];
    } else {
      const float2 w = tabt[64 * (o + j)];
      dst[addr(j)] = CONJ ? cmulc(w, v[j]) : cmul(v[j], w);
    }
  }
}

// Exchange barrier of one sequence.  Row mapping: the sequence's 64 threads are the two warps
// 2r, 2r + 1 (r = threadIdx.x / 64, at most 8 rows per CTA), which sync alone on named barrier
// 1 + r, so the rows of a CTA do not wait for each other.  Column mapping: every warp holds lanes
// of every column, so the whole CTA syncs.
template <bool ROW>
__device__ __forceinline__ void seq512_bar() {
  if constexpr (ROW) asm volatile("bar.sync %0, 64;" ::"r"(1 + (int)(threadIdx.x >> 6)) : "memory");
  else __syncthreads();
}

// Forward transform of one zero-padded sequence.  Entry: v[n1] = x[64 n1 + t] for n1 < 4.
// Exit: v[j2] = X[hi + 8 lo + 64 j2].  s0, s1: the sequence's two exchange buffers; tabt: the
// thread's twiddle row.  Contains two exchange barriers (seq512_bar).
template <bool ROW>
__device__ __forceinline__ void fwd512_zhi(float2 (&v)[8], float2* s0, float2* s1, int t, const float2* tabt) {
  using L = Lay512<ROW>;
  const int lo = t & 7, hi = t >> 3;
  dft8_lowhalf<false>(v);
  tw512_apply<false, true>(v, tabt, 0, s0, [&](int k1) { return L::y(t, k1); });
  seq512_bar<ROW>();
#pragma unroll
  for (int m1 = 0; m1 < 8; ++m1) v[m1] = s0[L::y(8 * m1 + lo, hi)];
  dft_pow2<8, false>(v);
  tw512_apply<false, true>(v, tabt, 8, s1, [&](int j1) { return L::v(hi, lo, j1); });
  seq512_bar<ROW>();
#pragma unroll
  for (int m2 = 0; m2 < 8; ++m2) v[m2] = s1[L::v(hi, m2, lo)];
  dft_pow2<8, false>(v);
}

// Inverse transform, first half of the output.  Entry: v[d2] = P[hi + 8 lo + 64 d2].
// Exit: v[e2] = y[t + 64 e2] for e2 < 4 (v[4..7] are not formed).  Contains two exchange
// barriers (seq512_bar).
template <bool ROW>
__device__ __forceinline__ void inv512_hout(float2 (&v)[8], float2* s0, float2* s1, int t, const float2* tabt) {
  using L = Lay512<ROW>;
  const int lo = t & 7, hi = t >> 3;
  dft_pow2<8, true>(v);
  tw512_apply<true, true>(v, tabt, 8, s0, [&](int e0) { return L::v(hi, lo, e0); });
  seq512_bar<ROW>();
#pragma unroll
  for (int d1 = 0; d1 < 8; ++d1) v[d1] = s0[L::v(hi, d1, lo)];
  dft_pow2<8, true>(v);
  tw512_apply<true, false>(v, tabt, 16, s1, [&](int e1) { return L::z(hi, lo, e1); });  // w^{d0 (e0 + 8 e1)}
  seq512_bar<ROW>();
#pragma unroll
  for (int d0 = 0; d0 < 8; ++d0) v[d0] = s1[L::z(d0, lo, hi)];
  dft_pow2<8, true>(v);
}

// Column pass for 2H = 512: T[:, kw] (rows < 256) = rows < 256 of IFFT(psf_hat[:, kw] FFT(T[:, kw]
// padded)).  CTA (g, y) transforms columns 8 g .. 8 g + 7 of the coil images y kTpImages ..
// (y + 1) kTpImages - 1 in turn; lanes run over the 8 columns first (row segments of 64 bytes),
// and blockIdx.x fastest keeps the CTAs in flight on whole rows of a few images.  The group's
// PSF columns (the same for every coil image) are read into shared memory once per CTA.
constexpr int kC5 = 8;          // columns per CTA
constexpr int kS5 = 514;        // exchange stride of one column (float2)
constexpr int kTpImages = 8;    // coil images per CTA
// exchange buffers, per-thread PSF slots (8 values), twiddle table
int smem_cols512() { return (2 * kC5 * kS5 + 8 * 64 * kC5 + kTwTab) * (int)sizeof(float2); }

__global__ void __launch_bounds__(64 * kC5, 2) k_tp_cols512(int BC, int W2, float2* __restrict__ T,
                                                           const float2* __restrict__ tw,
                                                           const float2* __restrict__ psf_hat) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int kT = 64 * kC5;
  const int c = threadIdx.x & (kC5 - 1), t = threadIdx.x / kC5;
  const int lo = t & 7, hi = t >> 3;
  float2* const base = reinterpret_cast<float2*>(smem);
  float2* tab = base + 2 * kC5 * kS5 + 8 * kT;
  float2* s0 = base + c * kS5;
  float2* s1 = s0 + kC5 * kS5;
  float2* ps = base + 2 * kC5 * kS5 + threadIdx.x;  // PSF slot j at ps[kT j]
  const float2* tabt = tab + t;
  const int col = blockIdx.x * kC5 + c;
  const bool live = col < W2;
  const int bc0 = blockIdx.y * kTpImages, bc1 = min(BC, bc0 + kTpImages);
  tw_copy(tab, tw, kTwTab);
#pragma unroll
  for (int j2 = 0; j2 < 8; ++j2)  // this thread's PSF values: k = hi + 8 lo + 64 j2
    ps[kT * j2] = live ? psf_hat[(size_t)(hi + 8 * lo + 64 * j2) * W2 + col] : make_float2(0.f, 0.f);
  __syncthreads();
  for (int bc = bc0; bc < bc1; ++bc) {
    float2* Tc = T + (size_t)bc * 256 * W2 + col;  // column col of image bc, rows < 256
    float2 v[8];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) v[n1] = live ? Tc[(size_t)(t + 64 * n1) * W2] : make_float2(0.f, 0.f);
    fwd512_zhi<false>(v, s0, s1, t, tabt);
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) v[j2] = cmul(v[j2], ps[kT * j2]);
    inv512_hout<false>(v, s0, s1, t, tabt);
    if (live) {
#pragma unroll
      for (int e2 = 0; e2 < 4; ++e2) Tc[(size_t)(t + 64 * e2) * W2] = v[e2];
    }
  }
}

// Row passes for 2W = 512, 8 rows per CTA (64 threads each, lanes along the row).
constexpr int kR5 = 8;
int smem_rows512() { return (2 * kR5 * 512 + kTwTab) * (int)sizeof(float2); }

// T[b,c,h,:] = FFT_512(S_c x [b,h,0..255], zero-padded).
__global__ void __launch_bounds__(64 * kR5, 2) k_tp_rows_fwd512(int C, int H, const float2* __restrict__ x,
                                                               const float2* __restrict__ maps,
                                                               float2* __restrict__ T,
                                                               const float2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int bc = blockIdx.y, b = bc / C;
  const int h = blockIdx.x * kR5 + r;
  const bool live = h < H;
  float2* const base = reinterpret_cast<float2*>(smem);
  float2* tab = base + 2 * kR5 * 512;
  float2* s0 = base + r * 512;
  float2* s1 = s0 + kR5 * 512;
  const size_t mrow = ((size_t)bc * H + h) * 256, xrow = ((size_t)b * H + h) * 256;
  tw_copy(tab, tw, kTwTab);
  float2 v[8];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1)
    v[n1] = live ? cmul(maps[mrow + t + 64 * n1], x[xrow + t + 64 * n1]) : make_float2(0.f, 0.f);
  __syncthreads();
  fwd512_zhi<true>(v, s0, s1, t, tab + t);
  if (live) {
    float2* Tr = T + ((size_t)bc * H + h) * 512 + (t >> 3) + 8 * (t & 7);
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) Tr[64 * j2] = v[j2];
  }
}

// out[b,h,:] = sum_c conj(S_c) IFFT_512(T[b,c,h,:])[0..255] + lambda x, the coils of group
// blockIdx.z (cpg < C: the partial sum goes to the first 256 entries of the rows of the group's
// first coil, as in k_tp_rows_inv).  The next coil's row is loaded into registers while the
// current one is transformed.
__global__ void __launch_bounds__(64 * kR5, 2) k_tp_rows_inv512(int C, int H, float2* __restrict__ T,
                                                               const float2* __restrict__ maps,
                                                               float2* __restrict__ out,
                                                               const float2* __restrict__ tw,
                                                               const float2* __restrict__ xin, float lam_host,
                                                               const double* __restrict__ lam_dev, int cpg,
                                                               double* __restrict__ dpart) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int b = blockIdx.y;
  const int h = blockIdx.x * kR5 + r;
  const bool live = h < H;
  float2* const base = reinterpret_cast<float2*>(smem);
  float2* tab = base + 2 * kR5 * 512;
  float2* s0 = base + r * 512;
  float2* s1 = s0 + kR5 * 512;
  const float2* tabt = tab + t;
  const int c0 = blockIdx.z * cpg, c1 = min(C, c0 + cpg);
  tw_copy(tab, tw, kTwTab);
  const int kin = (t >> 3) + 8 * (t & 7);  // this thread's input index k = hi + 8 lo (+ 64 d2)
  float2 nx[8], acc[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) acc[e] = make_float2(0.f, 0.f);
  auto fetch = [&](int c) {
    const float2* src = T + (((size_t)b * C + c) * H + h) * 512 + kin;
#pragma unroll
    for (int d2 = 0; d2 < 8; ++d2) nx[d2] = live ? src[64 * d2] : make_float2(0.f, 0.f);
  };
  fetch(c0);
  __syncthreads();  // twiddle table
  for (int c = c0; c < c1; ++c) {
    float2 v[8];
#pragma unroll
    for (int d2 = 0; d2 < 8; ++d2) v[d2] = nx[d2];
    if (c + 1 < c1) fetch(c + 1);
    inv512_hout<true>(v, s0, s1, t, tabt);
    if (live) {
      const float2* sm = maps + (((size_t)b * C + c) * H + h) * 256 + t;
#pragma unroll
      for (int e2 = 0; e2 < 4; ++e2) acc[e2] = cfmac(sm[64 * e2], v[e2], acc[e2]);
    }
  }
  if (!live) return;
  if (cpg < C) {
    float2* dst = T + (((size_t)b * C + c0) * H + h) * 512 + t;
#pragma unroll
    for (int e2 = 0; e2 < 4; ++e2) dst[64 * e2] = acc[e2];
    return;
  }
  const float lam = lam_dev ? (float)lam_dev[b] : lam_host;
  const size_t o = ((size_t)b * H + h) * 256 + t;
  float dot = 0.f;
#pragma unroll
  for (int e2 = 0; e2 < 4; ++e2) {
    const float2 xv = xin[o + 64 * e2];
    const float2 q = make_float2(fmaf(lam, xv.x, acc[e2].x), fmaf(lam, xv.y, acc[e2].y));
    out[o + 64 * e2] = q;
    dot = fmaf(xv.x, q.x, fmaf(xv.y, q.y, dot));
  }
  if (dpart) {  // Re<x, out> of this row, one slot per warp of the row (float-float warp sum, FP64 once)
    const float2 d = warp_sum_ff(dot);
    if ((threadIdx.x & 31) == 0) dpart[((size_t)b * H + h) * 2 + ((threadIdx.x >> 5) & 1)] = ff_to_d(d);
  }
}

// With cpg < C, CTA z sums coils z cpg .. z cpg + cpg - 1 and writes that partial sum over the
// first W entries of the rows of coil z cpg it has just read; k_coil_groups_sum (row stride 2W)
// adds the groups in fixed order and + lambda x.  The rows of the next coil are copied into a
// third shared buffer (cp.async) while the current coil is transformed.
template <int CLS>
__global__ void __launch_bounds__(kThreads, 2) k_tp_rows_inv(int C, int H, int W, float2* T,
                                                          const float2* maps, float2* out, Fft1DDev f,
                                                          const float2* xin, float lam_host,
                                                          const double* lam_dev, int cpg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W2 = f.L;
  float2* const base = reinterpret_cast<float2*>(smem);  // three buffers of kRows x W2
  const int bstride = kRows * W2;
  const int b = blockIdx.y;
  const int h0 = blockIdx.x * kRows;
  const int nr = min(kRows, H - h0);
  const int c0 = blockIdx.z * cpg, c1 = min(C, c0 + cpg);
  const int n16 = nr * W2 / 2;  // 16-byte chunks of one coil's rows (W2 even)
  auto fetch = [&](int c, float2* dst) {
    const float2* src = T + (((size_t)b * C + c) * H + h0) * W2;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) tp_cp_async16(dst + 2 * i, src + 2 * i);
    tp_cp_async_commit();
  };
  float2 acc[kMaxPer];
#pragma unroll
  for (int e = 0; e < kMaxPer; ++e) acc[e] = make_float2(0.f, 0.f);
  int ip = 0, is = 1, iq = 2;  // prefetched input, FFT scratch, next prefetch
  fetch(c0, base + ip * bstride);
  for (int c = c0; c < c1; ++c) {
    tp_cp_async_wait_all();
    __syncthreads();
    if (c + 1 < c1) fetch(c + 1, base + iq * bstride);
    float2* res = fft_smem_half<true, CLS, false, true>(base + ip * bstride, base + is * bstride, nr, f, W2);
#pragma unroll
    for (int e = 0; e < kMaxPer; ++e) {
      const int i = threadIdx.x + e * blockDim.x;  // output element (row r, column w < W)
      if (i < nr * W) {
        const int r = i / W, w = i - r * W;
        const float2 sm = maps[(((size_t)b * C + c) * H + h0 + r) * W + w];
        acc[e] = cfmac(sm, res[r * W2 + w], acc[e]);
      }
    }
    __syncthreads();
    const int t = ip;
    ip = iq;
    iq = t;
  }
  if (cpg < C) {  // partial sum of this coil group over the rows of coil c0 (already read)
#pragma unroll
    for (int e = 0; e < kMaxPer; ++e) {
      const int i = threadIdx.x + e * blockDim.x;
      if (i < nr * W) {
        const int r = i / W, w = i - r * W;
        T[(((size_t)b * C + c0) * H + h0 + r) * W2 + w] = acc[e];
      }
    }
    return;
  }
  const float lam = lam_dev ? (float)lam_dev[b] : lam_host;
#pragma unroll
  for (int e = 0; e < kMaxPer; ++e) {
    const int i = threadIdx.x + e * blockDim.x;
    if (i < nr * W) {
      const size_t o = ((size_t)b * H + h0) * W + i;
      const float2 xv = xin[o];
      out[o] = make_float2(fmaf(lam, xv.x, acc[e].x), fmaf(lam, xv.y, acc[e].y));
    }
  }
}

// ------------------------------------ Bluestein row passes of the normal operator
// A W-point DFT of a row (128 < W <= 256) as a 512-point circular convolution (Bluestein):
// with the chirp c_n = e^{s pi i n^2 / W} (s = -1 forward, +1 inverse; n^2 reduced mod 2W in
// integers on the host),
//   X_k = c_k sum_n (x_n c_n) conj(c_{k-n}) = c_k IFFT_512(FFT_512(a) . Bh)_k,   k < W,
// a = x c zero-padded to 512, Bh = FFT_512(b) / 512, b_m = conj(c_m) for |m| < W wrapped modulo
// 512 (2W - 1 <= 512: the circular convolution does not alias into k < W).  Both transforms
// are the register-resident ones above (input below 256, output below 256).  The plan's table
// block (sense_plan_s::blue) holds the two chirps [256] and the two spectra [512],
// each spectrum permuted so that the thread t holding k = hi + 8 lo + 64 j2 reads slot t + 64 j2.
constexpr int kRB = 4;  // rows per CTA (four 256-thread CTAs per SM)
constexpr int kBlueCf = 0, kBlueCi = 256, kBlueBf = 512, kBlueBi = 1024, kBlueN = 1536;
// exchange buffers, twiddle table, the pass's spectrum [512] and chirp [256]
int smem_blue() { return (2 * kRB * 512 + kTwTab + 512 + 256) * (int)sizeof(float2); }

__device__ __forceinline__ void blue_tables(float2* bh, float2* ch, const float2* __restrict__ Bh,
                                            const float2* __restrict__ chirp) {
  for (int i = threadIdx.x; i < 512; i += blockDim.x) bh[i] = __ldg(Bh + i);
  for (int i = threadIdx.x; i < 256; i += blockDim.x) ch[i] = __ldg(chirp + i);
}

// T[b,c,h,k] = sum_n S_c x [b,h,n] e^{-2 pi i n k / W}  (the plain row DFT of the normal operator)
__global__ void __launch_bounds__(64 * kRB, 4) k_blue_rows_fwd(int C, int H, int W, const float2* __restrict__ x,
                                                              const float2* __restrict__ maps,
                                                              float2* __restrict__ T,
                                                              const float2* __restrict__ tw,
                                                              const float2* __restrict__ blue) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int bc = blockIdx.y, b = bc / C;
  const int h = blockIdx.x * kRB + r;
  const bool live = h < H;
  float2* const base = reinterpret_cast<float2*>(smem);
  float2* s0 = base + r * 512;
  float2* s1 = s0 + kRB * 512;
  float2* tab = base + 2 * kRB * 512;
  float2* bh = tab + kTwTab;
  float2* ch = bh + 512;
  tw_copy(tab, tw, kTwTab);
  blue_tables(bh, ch, blue + kBlueBf, blue + kBlueCf);
  const size_t row = ((size_t)bc * H + h) * W, xrow = ((size_t)b * H + h) * W;
  float2 v[8];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    const int n = t + 64 * n1;
    v[n1] = (live && n < W) ? cmul(maps[row + n], x[xrow + n]) : make_float2(0.f, 0.f);
  }
  __syncthreads();
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) v[n1] = cmul(v[n1], ch[t + 64 * n1]);
  fwd512_zhi<true>(v, s0, s1, t, tab + t);
#pragma unroll
  for (int j2 = 0; j2 < 8; ++j2) v[j2] = cmul(v[j2], bh[t + 64 * j2]);
  inv512_hout<true>(v, s0, s1, t, tab + t);
  if (live) {
#pragma unroll
    for (int e2 = 0; e2 < 4; ++e2) {
      const int k = t + 64 * e2;
      if (k < W) T[row + k] = cmul(v[e2], ch[k]);
    }
  }
}

// out[b,h,n] = sum_c conj(S_c) sum_k T[b,c,h,k] e^{+2 pi i n k / W} + lambda x over the coils of
// group blockIdx.z (cpg < C: the partial sum goes to the row of the group's first coil in T, for
// k_coil_groups_sum).
__global__ void __launch_bounds__(64 * kRB, 4) k_blue_rows_inv(int C, int H, int W, float2* __restrict__ T,
                                                              const float2* __restrict__ maps,
                                                              float2* __restrict__ out,
                                                              const float2* __restrict__ tw,
                                                              const float2* __restrict__ blue,
                                                              const float2* __restrict__ xin, float lam_host,
                                                              const double* __restrict__ lam_dev, int cpg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int b = blockIdx.y;
  const int h = blockIdx.x * kRB + r;
  const bool live = h < H;
  float2* const base = reinterpret_cast<float2*>(smem);
  float2* s0 = base + r * 512;
  float2* s1 = s0 + kRB * 512;
  float2* tab = base + 2 * kRB * 512;
  float2* bh = tab + kTwTab;
  float2* ch = bh + 512;
  const int c0 = blockIdx.z * cpg, c1 = min(C, c0 + cpg);
  tw_copy(tab, tw, kTwTab);
  blue_tables(bh, ch, blue + kBlueBi, blue + kBlueCi);
  float2 nx[4], acc[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) acc[e] = make_float2(0.f, 0.f);
  auto fetch = [&](int c) {
    const float2* src = T + (((size_t)b * C + c) * H + h) * W;
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
      const int k = t + 64 * n1;
      nx[n1] = (live && k < W) ? src[k] : make_float2(0.f, 0.f);
    }
  };
  __syncthreads();  // tables
  for (int c = c0; c < c1; ++c) {
    float2 v[8];
    fetch(c);
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) v[n1] = cmul(nx[n1], ch[t + 64 * n1]);
    fwd512_zhi<true>(v, s0, s1, t, tab + t);
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) v[j2] = cmul(v[j2], bh[t + 64 * j2]);
    inv512_hout<true>(v, s0, s1, t, tab + t);
    if (live) {
      const float2* sm = maps + (((size_t)b * C + c) * H + h) * W;
#pragma unroll
      for (int e2 = 0; e2 < 4; ++e2) {
        const int n = t + 64 * e2;
        if (n < W) acc[e2] = cfmac(sm[n], cmul(v[e2], ch[n]), acc[e2]);
      }
    }
  }
  if (!live) return;
  if (cpg < C) {
    float2* dst = T + (((size_t)b * C + c0) * H + h) * W;
#pragma unroll
    for (int e2 = 0; e2 < 4; ++e2) {
      const int n = t + 64 * e2;
      if (n < W) dst[n] = acc[e2];
    }
    return;
  }
  const float lam = lam_dev ? (float)lam_dev[b] : lam_host;
  const size_t o = ((size_t)b * H + h) * W;
#pragma unroll
  for (int e2 = 0; e2 < 4; ++e2) {
    const int n = t + 64 * e2;
    if (n < W) {
      const float2 xv = xin[o + n];
      out[o + n] = make_float2(fmaf(lam, xv.x, acc[e2].x), fmaf(lam, xv.y, acc[e2].y));
    }
  }
}

// ------------------------------------ direct row passes for W = 8 P (P prime, 17 <= P <= 31)
// A row of W = 8 P points per warp.  With n = t + P n1 and k = k1 + 8 k2 (w = e^{-2 pi i / W}):
//   forward   X[k1 + 8 k2] = sum_t w_P^{t k2} Y[k1][t],  Y[k1][t] = w^{t k1} sum_{n1} x[t + P n1] w_8^{n1 k1}
//   inverse   x[t + P n1] = sum_{k1} w_8^{-n1 k1} Z[k1][t],  Z[k1][t] = w^{-t k1} sum_{k2} X[k1 + 8 k2] w_P^{-t k2}
// The 8-point DFTs run in registers (lane t < P); the P-point DFTs are direct sums over the
// conjugate pairs (t, P - t), S = a_t + a_{P-t}, D = a_t - a_{P-t}:
//   sum_t a_t w_P^{+-t k} = a_0 + sum_{t <= (P-1)/2} (S cos(2 pi t k / P) -+ i D sin(2 pi t k / P))
// so one cosine and sine give the outputs k and P - k.  Lane (k1 = lane & 7, g = lane >> 3)
// takes the output pairs g, g + 4, g + 8, ... <= (P-1)/2 of residue k1 (pair 0 is the single
// output 0).  Each lane keeps t k mod P incrementally and reads cos, sin from a P-entry table.
constexpr int kR8Rows = 8;  // rows (warps) per CTA
template <int P>
int smem_r8p() { return (32 + kR8Rows * 16 * P) * (int)sizeof(float2); }

// (cos, sin)(2 pi m / P) from the plan's W-point roots e^{-2 pi i m / W} at m 8.
template <int P>
__device__ __forceinline__ void r8p_cs(float2* cs, const float2* __restrict__ tw) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const float2 w = __ldg(tw + 8 * i);
    cs[i] = make_float2(w.x, -w.y);
  }
}

// P-point sums of one residue k1 over the pairs of this lane: za[q] = sum_t S_t cos - s D_t sin
// (SIGN = -1: forward; +1: inverse, i D s with the opposite sign), zb[q] the partner output P - k.
// get(t) returns a_t of the residue.
template <int P, int SIGN, typename Get>
__device__ __forceinline__ void r8p_pairs(int g, const float2* cs, Get get, float2 (&za)[4], float2 (&zb)[4]) {
  constexpr int HP = (P - 1) / 2;
  int m[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    za[q] = zb[q] = make_float2(0.f, 0.f);
    m[q] = 0;
  }
#pragma unroll 2
  for (int t = 1; t <= HP; ++t) {
    const float2 a = get(t), b = get(P - t);
    const float2 S = cadd(a, b), D = csub(a, b);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int it = g + 4 * q;  // pair index; t it mod P kept in m[q]
      m[q] += it;
      if (m[q] >= P) m[q] -= P;
      const float2 w = cs[it <= HP ? m[q] : 0];
      // forward: S c - i D s = (S.x c + D.y s, S.y c - D.x s); inverse: S c + i D s
      const float sy = SIGN < 0 ? D.y * w.y : -D.y * w.y, sx = SIGN < 0 ? -D.x * w.y : D.x * w.y;
      za[q].x = fmaf(S.x, w.x, za[q].x + sy);
      za[q].y = fmaf(S.y, w.x, za[q].y + sx);
      zb[q].x = fmaf(S.x, w.x, zb[q].x - sy);
      zb[q].y = fmaf(S.y, w.x, zb[q].y - sx);
    }
  }
}

// T[b,c,h,k] = sum_n S_c x [b,h,n] e^{-2 pi i n k / W}  (the plain row DFT of the normal operator)
template <int P>
__global__ void __launch_bounds__(32 * kR8Rows, 4) k_r8p_fwd(int C, int H, const float2* __restrict__ x,
                                                            const float2* __restrict__ maps,
                                                            float2* __restrict__ T,
                                                            const float2* __restrict__ tw) {
  constexpr int W = 8 * P, HP = (P - 1) / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* cs = reinterpret_cast<float2*>(smem);
  float2* Y = cs + 32 + warp * 16 * P;  // [8][P]
  r8p_cs<P>(cs, tw);
  __syncthreads();
  const int bc = blockIdx.y, b = bc / C, h = blockIdx.x * kR8Rows + warp;
  if (h >= H) return;  // whole warp, after the only CTA barrier
  const size_t row = ((size_t)bc * H + h) * W, xrow = ((size_t)b * H + h) * W;
  if (lane < P) {
    float2 v[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) v[n1] = cmul(maps[row + lane + P * n1], x[xrow + lane + P * n1]);
    dft_pow2<8, false>(v);
    Y[lane] = v[0];
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) Y[k1 * P + lane] = cmul(v[k1], __ldg(tw + lane * k1));
  }
  __syncwarp();
  const int k1 = lane & 7, g = lane >> 3;
  const float2* Yk = Y + k1 * P;
  float2 za[4], zb[4];
  r8p_pairs<P, -1>(g, cs, [&](int t) { return Yk[t]; }, za, zb);
  const float2 y0 = Yk[0];
  float2* Tr = T + row + k1;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int it = g + 4 * q;
    if (it <= HP) {
      Tr[8 * it] = cadd(y0, za[q]);
      if (it > 0) Tr[8 * (P - it)] = cadd(y0, zb[q]);
    }
  }
}

// out[b,h,n] = sum_c conj(S_c) sum_k T[b,c,h,k] e^{+2 pi i n k / W} + lambda x over the coils of
// group blockIdx.z (cpg < C: the partial sum goes to the row of the group's first coil in T, for
// k_coil_groups_sum).
template <int P>
__global__ void __launch_bounds__(32 * kR8Rows, 4) k_r8p_inv(int C, int H, float2* __restrict__ T,
                                                            const float2* __restrict__ maps,
                                                            float2* __restrict__ out,
                                                            const float2* __restrict__ tw,
                                                            const float2* __restrict__ xin, float lam_host,
                                                            const double* __restrict__ lam_dev, int cpg) {
  constexpr int W = 8 * P, HP = (P - 1) / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* cs = reinterpret_cast<float2*>(smem);
  float2* R = cs + 32 + warp * 16 * P;  // the coil's row [W]
  float2* Z = R + W;                    // [8][P]
  r8p_cs<P>(cs, tw);
  __syncthreads();
  const int b = blockIdx.y, h = blockIdx.x * kR8Rows + warp;
  if (h >= H) return;  // whole warp, after the only CTA barrier
  const int c0 = blockIdx.z * cpg, c1 = min(C, c0 + cpg);
  const int k1 = lane & 7, g = lane >> 3;
  float2 acc[8];
#pragma unroll
  for (int n1 = 0; n1 < 8; ++n1) acc[n1] = make_float2(0.f, 0.f);
  for (int c = c0; c < c1; ++c) {
    const size_t row = (((size_t)b * C + c) * H + h) * W;
    for (int i = lane; i < W; i += 32) R[i] = T[row + i];
    __syncwarp();
    float2 za[4], zb[4];
    r8p_pairs<P, 1>(g, cs, [&](int k2) { return R[k1 + 8 * k2]; }, za, zb);
    const float2 x0 = R[k1];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int it = g + 4 * q;
      if (it <= HP) {
        Z[k1 * P + it] = cmulc(__ldg(tw + it * k1), cadd(x0, za[q]));
        if (it > 0) Z[k1 * P + P - it] = cmulc(__ldg(tw + (P - it) * k1), cadd(x0, zb[q]));
      }
    }
    __syncwarp();
    if (lane < P) {
      float2 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = Z[j * P + lane];
      dft_pow2<8, true>(v);
      const float2* sm = maps + row + lane;
#pragma unroll
      for (int n1 = 0; n1 < 8; ++n1) acc[n1] = cfmac(sm[P * n1], v[n1], acc[n1]);
    }
    __syncwarp();
  }
  if (lane >= P) return;
  if (cpg < C) {
    float2* dst = T + (((size_t)b * C + c0) * H + h) * W + lane;
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) dst[P * n1] = acc[n1];
    return;
  }
  const float lam = lam_dev ? (float)lam_dev[b] : lam_host;
  const size_t o = ((size_t)b * H + h) * W + lane;
#pragma unroll
  for (int n1 = 0; n1 < 8; ++n1) {
    const float2 xv = xin[o + P * n1];
    out[o + P * n1] = make_float2(fmaf(lam, xv.x, acc[n1].x), fmaf(lam, xv.y, acc[n1].y));
  }
}

// ------------------------------------ column pass of the normal operator for H = 256
// dst = IDFT_256(m2s . DFT_256(T[:, kw])) in place, the transforms held in registers: 32 threads
// per column, 8 points each, 256 = 8 x 8 x 4, two shared exchanges per transform.  Digits
// (w = e^{-2 pi i / 256}; thread t = lo + 4 hi of its column, lo < 4, hi < 8):
//   forward, n = 32 n1 + n2:
//     s1  t = n2:              Y[n2][k1] = w^{n2 k1} sum_{n1} x[32 n1 + n2] w^{32 n1 k1}
//     s2  t = m2 + 4 k1:       V[k1][m2][j1] = w^{8 m2 j1} sum_{m1} Y[4 m1 + m2][k1] w^{32 m1 j1}
//     s3  t = a + 4 k1, j1 in {a, a + 4}:  X[k1 + 8 j1 + 64 j2] = sum_{m2} V[k1][m2][j1] w^{64 m2 j2}
//   the mask product where s3 leaves X; the inverse in decimation-in-frequency order from there
//   (k = d0 + 8 d1 + 64 d2, n = e0 + 4 e1 + 32 e2):
//     A   t = a + 4 d0, d1 in {a, a + 4}:  U[d0][d1][e0] = w^{-8 e0 d1} sum_{d2} P[k] w^{-64 d2 e0}
//     B   t = e0 + 4 d0:       Z[d0][e0][e1] = w^{-d0 (e0 + 4 e1)} sum_{d1} U[d0][d1][e0] w^{-32 d1 e1}
//     C   t = e0 + 4 e1:       y[e0 + 4 e1 + 32 e2] = sum_{d0} Z[d0][e0][e1] w^{-32 d0 e2}
// Lanes run over 8 columns first; with the column stride 258 (2 mod 16) and the layouts of Y,
// V, U, Z below, the 16 lanes of every half-warp access 16 different bank pairs.
constexpr int kC6 = 8;           // columns per CTA
constexpr int kS6 = 258;         // exchange stride of one column (float2)
constexpr int kCol256Images = 4; // coil images per CTA
constexpr int kTw256 = 32;       // twiddle slots per thread index
// exchange buffers, twiddle table, per-thread mask slots (8 floats)
int smem_col256() { return (2 * kC6 * kS6 + kTw256 * 32 + 4 * 32 * kC6) * (int)sizeof(float2); }

__device__ __forceinline__ int l256_y(int n2, int k1) { return 32 * k1 + n2; }
__device__ __forceinline__ int l256_v(int k1, int m2, int j1) { return 32 * k1 + 8 * m2 + ((j1 + m2) & 7); }
__device__ __forceinline__ int l256_u(int d0, int d1, int e0) { return 32 * d0 + 4 * d1 + ((e0 + d1) & 3); }

// slots: 0..7 w^{t k1}; 8..15 w^{8 lo j1}; 16 + 4 q + e0: w^{8 e0 (lo + 4 q)}; 24 + e1:
// w^{hi (lo + 4 e1)}; exponent of slot s of thread t in units of 2 pi / 256 (the plan holds the
// table at sense_plan_s::twtab + kTwTab, slot-major)
SENSE_HD int tw256_exp(int s, int t) {
  const int lo = t & 3, hi = t >> 2;
  int e;
  if (s < 8) e = t * s;
  else if (s < 16) e = 8 * lo * (s - 8);
  else if (s < 24) e = 8 * ((s - 16) & 3) * (lo + 4 * ((s - 16) >> 2));
  else e = hi * (lo + 4 * (s - 24));
  return e & 255;
}

__global__ void __launch_bounds__(32 * kC6, 4) k_col256(int BC, int W, float2* __restrict__ T,
                                                       const float2* __restrict__ tw,
                                                       const float* __restrict__ m2s, int lines) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int c = threadIdx.x & (kC6 - 1), t = threadIdx.x / kC6;
  const int lo = t & 3, hi = t >> 2;
  float2* const base = reinterpret_cast<float2*>(smem);
  float2* s0 = base + c * kS6;
  float2* s1 = s0 + kC6 * kS6;
  float2* tab = base + 2 * kC6 * kS6;
  const float2* tt = tab + t;  // slot s at tt[32 s]
  const int col = blockIdx.x * kC6 + c;
  const bool live = col < W;
  float* mk = reinterpret_cast<float*>(tab + kTw256 * 32) + threadIdx.x;  // slot 4 q + j2 at mk[32 kC6 (4 q + j2)]
  tw_copy(tab, tw, kTw256 * 32);
#pragma unroll
  for (int q = 0; q < 2; ++q)  // mask^2/(HW) at k = hi + 8 (lo + 4 q) + 64 j2
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2)
      mk[32 * kC6 * (4 * q + j2)] =
          live ? __ldg(m2s + (lines ? col : (size_t)(hi + 8 * (lo + 4 * q) + 64 * j2) * W + col)) : 0.f;
  __syncthreads();
  const int bc0 = blockIdx.y * kCol256Images, bc1 = min(BC, bc0 + kCol256Images);
  for (int bc = bc0; bc < bc1; ++bc) {
    float2* Tc = T + (size_t)bc * 256 * W + col;
    float2 v[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) v[n1] = live ? Tc[(size_t)(t + 32 * n1) * W] : make_float2(0.f, 0.f);
    dft_pow2<8, false>(v);
    s0[l256_y(t, 0)] = v[0];
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) s0[l256_y(t, k1)] = cmul(v[k1], tt[32 * k1]);
    __syncthreads();
#pragma unroll
    for (int m1 = 0; m1 < 8; ++m1) v[m1] = s0[l256_y(4 * m1 + lo, hi)];
    dft_pow2<8, false>(v);
    s1[l256_v(hi, lo, 0)] = v[0];
#pragma unroll
    for (int j1 = 1; j1 < 8; ++j1) s1[l256_v(hi, lo, j1)] = cmul(v[j1], tt[32 * (8 + j1)]);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float2 u[4];
#pragma unroll
      for (int m2 = 0; m2 < 4; ++m2) u[m2] = s1[l256_v(hi, m2, lo + 4 * q)];
      dft_pow2<4, false>(u);
#pragma unroll
      for (int j2 = 0; j2 < 4; ++j2) u[j2] = cscale(u[j2], mk[32 * kC6 * (4 * q + j2)]);
      dft_pow2<4, true>(u);
      s0[l256_u(hi, lo + 4 * q, 0)] = u[0];
#pragma unroll
      for (int e0 = 1; e0 < 4; ++e0) s0[l256_u(hi, lo + 4 * q, e0)] = cmulc(tt[32 * (16 + 4 * q + e0)], u[e0]);
    }
    __syncthreads();
#pragma unroll
    for (int d1 = 0; d1 < 8; ++d1) v[d1] = s0[l256_u(hi, d1, lo)];
    dft_pow2<8, true>(v);
#pragma unroll
    for (int e1 = 0; e1 < 8; ++e1) s1[lo + 4 * e1 + 32 * hi] = cmulc(tt[32 * (24 + e1)], v[e1]);
    __syncthreads();
#pragma unroll
    for (int d0 = 0; d0 < 8; ++d0) v[d0] = s1[t + 32 * d0];
    dft_pow2<8, true>(v);
    if (live) {
#pragma unroll
      for (int e2 = 0; e2 < 8; ++e2) Tc[(size_t)(t + 32 * e2) * W] = v[e2];
    }
  }
}

// psf_hat = FFT2(psf) / (4 H W): rows along 2W, then columns along 2H (in place, one array).
template <int CLS>
__global__ void __launch_bounds__(kThreads, 2) k_tp_psf_rows(int H2, const float2* psf, float2* out, Fft1DDev f) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W2 = f.L;
  float2* a = reinterpret_cast<float2*>(smem);
  float2* bb = a + kRows * W2;
  const int h0 = blockIdx.x * kRows;
  const int nr = min(kRows, H2 - h0);
  for (int i = threadIdx.x; i < nr * W2; i += blockDim.x) a[i] = psf[(size_t)h0 * W2 + i];
  __syncthreads();
  float2* res = fft_smem<false, CLS>(a, bb, nr, f, W2);
  for (int i = threadIdx.x; i < nr * W2; i += blockDim.x) out[(size_t)h0 * W2 + i] = res[i];
}

template <int CLS>
__global__ void __launch_bounds__(kThreads, 2) k_tp_psf_cols(int W2, float2* io, Fft1DDev f, float scale) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int H2 = f.L, ld = H2 + 1;
  float2* a = reinterpret_cast<float2*>(smem);
  float2* bb = a + kCols * ld;
  const int w0 = blockIdx.x * kCols;
  const int nc = min(kCols, W2 - w0);
  for (int i = threadIdx.x; i < H2 * kCols; i += blockDim.x) {
    const int h = i / kCols, cc = i - h * kCols;
    a[cc * ld + h] = cc < nc ? io[(size_t)h * W2 + w0 + cc] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* res = fft_smem<false, CLS>(a, bb, kCols, f, ld);
  for (int i = threadIdx.x; i < H2 * kCols; i += blockDim.x) {
    const int h = i / kCols, cc = i - h * kCols;
    if (cc < nc) io[(size_t)h * W2 + w0 + cc] = cscale(res[cc * ld + h], scale);
  }
}

// PSF of a non-Cartesian trajectory on the 2H x 2W grid (direct sum; products of FP32 phasors,
// FP64 accumulation):  psf[iy][ix] = (H W)^{-1} sum_m exp(2 pi i (ky_m dy / H + kx_m dx / W)),
// dy = iy (iy < H) or iy - 2H, likewise dx; zero on row H and column W.  One thread per grid point;
// the CTA's 16 x 16 block stages chunks of the trajectory and their phasors in shared memory.
constexpr int kPsfTile = 16, kPsfChunk = 64;
__global__ void __launch_bounds__(256) k_tp_psf(int M, int H, int W, const float* traj, float2* psf) {
  __shared__ float2 ey[kPsfChunk][kPsfTile], ex[kPsfChunk][kPsfTile];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int iy = blockIdx.y * kPsfTile + ty, ix = blockIdx.x * kPsfTile + tx;
  const int iy0 = blockIdx.y * kPsfTile, ix0 = blockIdx.x * kPsfTile;
  double re = 0.0, im = 0.0;
  for (int m0 = 0; m0 < M; m0 += kPsfChunk) {
    __syncthreads();
    for (int i = threadIdx.x; i < kPsfChunk * kPsfTile; i += blockDim.x) {
      const int mm = i / kPsfTile, j = i - mm * kPsfTile, m = m0 + mm;
      float2 vy = make_float2(0.f, 0.f), vx = vy;
      if (m < M) {
        const int gy = iy0 + j, gx = ix0 + j;
        const double dy = gy < H ? gy : gy - 2 * H, dx = gx < W ? gx : gx - 2 * W;
        // phase in turns, reduced to [0, 1) in FP64 before the FP32 sin/cos
        double ty_ = (double)traj[2 * m] * dy / H, tx_ = (double)traj[2 * m + 1] * dx / W;
        ty_ -= floor(ty_);
        tx_ -= floor(tx_);
        float sy, cy, sx, cx;
        sincospif(2.f * (float)ty_, &sy, &cy);
        sincospif(2.f * (float)tx_, &sx, &cx);
        vy = make_float2(cy, sy);
        vx = make_float2(cx, sx);
      }
      ey[mm][j] = vy;
      ex[mm][j] = vx;
    }
    __syncthreads();
    const int mmax = min(kPsfChunk, M - m0);
    for (int mm = 0; mm < mmax; ++mm) {
      const float2 p = cmul(ey[mm][ty], ex[mm][tx]);
      re += (double)p.x;
      im += (double)p.y;
    }
  }
  if (iy < 2 * H && ix < 2 * W) {
    const double sc = (iy == H || ix == W) ? 0.0 : 1.0 / ((double)H * W);
    psf[(size_t)iy * 2 * W + ix] = make_float2((float)(re * sc), (float)(im * sc));
  }
}

// Radix class of a 1-D plan (see fft_smem).
int fft_class(const Fft1D& f) {
  int cls = 0;
  for (int i = 0; i < f.nst; ++i) {
    const int r = f.radix[i];
    if (r == 3 || r == 5 || r == 7) cls = cls < 1 ? 1 : cls;
    else if (r != 2 && r != 4 && r != 8) cls = 2;
  }
  return cls;
}

#define SENSE_LAUNCH_CLS(cls, kernel, grid, smem_bytes, stream, ...)                       \
  do {                                                                                      \
    if ((cls) == 0) kernel<0><<<(grid), kThreads, (smem_bytes), (stream)>>>(__VA_ARGS__);   \
    else if ((cls) == 1) kernel<1><<<(grid), kThreads, (smem_bytes), (stream)>>>(__VA_ARGS__); \
    else kernel<2><<<(grid), kThreads, (smem_bytes), (stream)>>>(__VA_ARGS__);             \
  } while (0)

template <typename K>
bool set_smem3(K k0, K k1, K k2, int bytes) {
  return cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
         cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
         cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
}
#define SENSE_SET_SMEM(kernel, bytes) set_smem3(kernel<0>, kernel<1>, kernel<2>, (bytes))

Fft1DDev dev(const Fft1D& f) {
  Fft1DDev d;
  d.L = f.L;
  d.nst = f.nst;
  for (int i = 0; i < SENSE_MAX_STAGES; ++i) d.radix[i] = f.radix[i];
  d.tw = f.tw;
  return d;
}

bool set_smem(const void* k, int bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
}

int smem_rows(int W) { return 2 * kRows * W * (int)sizeof(float2); }
int smem_cols(int H) { return 2 * kCols * (H + 1) * (int)sizeof(float2); }

}  // namespace

// Factor L into radices 8, 4, 2 and odd primes <= 31; fill the twiddle table.
int build_fft1d(Fft1D& f, int L, std::vector<float2>& host_tw) {
  f.L = L;
  f.nst = 0;
  int n = L;
  while (n % 8 == 0 && f.nst < SENSE_MAX_STAGES) { f.radix[f.nst++] = 8; n /= 8; }
  while (n % 4 == 0 && f.nst < SENSE_MAX_STAGES) { f.radix[f.nst++] = 4; n /= 4; }
  while (n % 2 == 0 && f.nst < SENSE_MAX_STAGES) { f.radix[f.nst++] = 2; n /= 2; }
  const int primes[] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31};
  for (int p : primes)
    while (n % p == 0 && f.nst < SENSE_MAX_STAGES) { f.radix[f.nst++] = p; n /= p; }
  if (n != 1) return SENSE_EUNSUPPORTED;
  host_tw.resize(L);
  for (int m = 0; m < L; ++m) {
    const double ang = -2.0 * M_PI * m / L;
    host_tw[m] = make_float2((float)cos(ang), (float)sin(ang));
  }
  return SENSE_OK;
}

// Column pass of the normal operator over p->w.T [B][C][H][W]: IDFT_H(m2s . DFT_H), in place
// (register-resident for H = 256, else the generic k_col; the map sets are already summed in T).
bool use_col256(sense_plan p) { return p->H == 256 && !p->toep; }

// Per-thread-index twiddle tables of the register-resident transforms (slot-major, FP64 on the
// host): the 512-point table at twtab, the 256-point one at twtab + kTwTab.
int twtab_prepare(sense_plan p) {
  if (p->twtab) return SENSE_OK;
  std::vector<float2> h(kTwTab + kTw256 * 32);
  for (int i = 0; i < kTwTab; ++i) {
    const double a = -2.0 * M_PI * tw512_exp(i >> 6, i & 63) / 512.0;
    h[i] = make_float2((float)cos(a), (float)sin(a));
  }
  for (int i = 0; i < kTw256 * 32; ++i) {
    const double a = -2.0 * M_PI * tw256_exp(i >> 5, i & 31) / 256.0;
    h[kTwTab + i] = make_float2((float)cos(a), (float)sin(a));
  }
  if (cudaMalloc(&p->twtab, h.size() * sizeof(float2)) != cudaSuccess) {
    p->twtab = nullptr;
    return SENSE_ECUDA;
  }
  return cudaMemcpy(p->twtab, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess
             ? SENSE_OK
             : SENSE_ECUDA;
}

// The normal operator's row passes are direct for W = 8 P (P prime, 17 .. 31); else they go
// through Bluestein's 512-point convolution where the generic transform would need a radix
// above 7 (class 2) and 2W - 1 <= 512.
int r8p_of(sense_plan p) {
  if (p->S != 1 || p->toep || p->W % 8) return 0;
  const int P = p->W / 8;
  return (P == 17 || P == 19 || P == 23 || P == 29 || P == 31) ? P : 0;
}
bool use_blue(sense_plan p) {
  return !r8p_of(p) && p->S == 1 && !p->toep && p->W > 128 && p->W <= 256 && fft_class(p->fW) == 2;
}

#define SENSE_R8P_SWITCH(P, ...)                              \
  switch (P) {                                                 \
    case 17: { constexpr int kP = 17; __VA_ARGS__; } break;    \
    case 19: { constexpr int kP = 19; __VA_ARGS__; } break;    \
    case 23: { constexpr int kP = 23; __VA_ARGS__; } break;    \
    case 29: { constexpr int kP = 29; __VA_ARGS__; } break;    \
    case 31: { constexpr int kP = 31; __VA_ARGS__; } break;    \
    default: break;                                            \
  }

int r8p_prepare(sense_plan p) {
  const int P = r8p_of(p);
  bool ok = true;
  SENSE_R8P_SWITCH(P, ok = cudaFuncSetAttribute(k_r8p_fwd<kP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                smem_r8p<kP>()) == cudaSuccess &&
                           cudaFuncSetAttribute(k_r8p_inv<kP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                smem_r8p<kP>()) == cudaSuccess)
  if (!ok) return SENSE_ECUDA;
  p->r8p = P;
  return SENSE_OK;
}

// Bluestein tables (layout kBlue*), FP64 on the host with the phases reduced in integers.
int blue_prepare(sense_plan p) {
  const int W = p->W, L = 512;
  std::vector<float2> h(kBlueN, make_float2(0.f, 0.f));
  std::vector<double> rc(L), rs(L);
  for (int m = 0; m < L; ++m) {
    rc[m] = cos(2.0 * M_PI * m / L);
    rs[m] = -sin(2.0 * M_PI * m / L);  // e^{-2 pi i m / L}
  }
  for (int si = 0; si < 2; ++si) {
    const double sg = si == 0 ? -1.0 : 1.0;  // forward, inverse
    std::vector<double> br(L, 0.0), bi(L, 0.0);
    for (int n = 0; n < W; ++n) {
      const double ang = M_PI * (double)(((long long)n * n) % (2 * W)) / W;  // pi n^2 / W
      h[(si == 0 ? kBlueCf : kBlueCi) + n] = make_float2((float)cos(ang), (float)(sg * sin(ang)));
      br[n] = cos(ang);        // b_n = conj(c_n)
      bi[n] = -sg * sin(ang);
      if (n > 0) {
        br[L - n] = br[n];
        bi[L - n] = bi[n];
      }
    }
    for (int k = 0; k < L; ++k) {  // Bh_k = sum_m b_m e^{-2 pi i m k / L} / L
      double xr = 0.0, xi = 0.0;
      for (int m = 0; m < L; ++m) {
        const int e = (int)(((long long)m * k) % L);
        xr += br[m] * rc[e] - bi[m] * rs[e];
        xi += br[m] * rs[e] + bi[m] * rc[e];
      }
      // stored at the index of the thread that reads it: thread t = lo + 8 hi holds
      // k = hi + 8 lo + 64 j2 after the forward transform and reads slot t + 64 j2
      const int j2 = k >> 6, hi = k & 7, lo = (k >> 3) & 7;
      h[(si == 0 ? kBlueBf : kBlueBi) + lo + 8 * hi + 64 * j2] = make_float2((float)(xr / L), (float)(xi / L));
    }
  }
  if (cudaMalloc(&p->blue, kBlueN * sizeof(float2)) != cudaSuccess) {
    p->blue = nullptr;
    return SENSE_ECUDA;
  }
  if (cudaMemcpy(p->blue, h.data(), kBlueN * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaFuncSetAttribute(k_blue_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_blue()) != cudaSuccess ||
      cudaFuncSetAttribute(k_blue_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_blue()) != cudaSuccess)
    return SENSE_ECUDA;
  return SENSE_OK;
}

int generic_prepare(sense_plan p) {
  if (kRows * p->W > kThreads * kMaxPer) return SENSE_EUNSUPPORTED;
  const int sr = smem_rows(p->W), sc = smem_cols(p->H);
  if (sr > 200 * 1024 || sc > 200 * 1024) return SENSE_EUNSUPPORTED;
  if (!SENSE_SET_SMEM(k_row_expand, sr) || !SENSE_SET_SMEM(k_row_combine, smem_rows_inv(p->W)) ||
      !SENSE_SET_SMEM(k_col, sc))
    return SENSE_ECUDA;
  if (use_col256(p) && cudaFuncSetAttribute(k_col256, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            smem_col256()) != cudaSuccess)
    return SENSE_ECUDA;
  if (use_col256(p) || use_blue(p))
    if (int e = twtab_prepare(p)) return e;
  if (r8p_of(p)) return r8p_prepare(p);
  if (use_blue(p)) return blue_prepare(p);
  return SENSE_OK;
}

// Row pass with coil combination over p->w.T.  Few row tiles (small batches) leave most SMs idle
// while each CTA walks all coils, so with one map set the coils are split into groups across
// grid.z (about 1024 CTAs in all) and the group sums are added by a second, streaming kernel.
int launch_row_combine(sense_plan p, float2* out, int mode, const float2* xin, float lam_host,
                       const double* lam_dev) {
  const int nrb = (p->H + kRows - 1) / kRows;
  int groups = 1;
  if (p->S == 1) {
    groups = (1024 + nrb * p->B - 1) / (nrb * p->B);
    groups = groups < 1 ? 1 : (groups > p->C ? p->C : groups);
  }
  const int cpg = (p->C + groups - 1) / groups;
  groups = (p->C + cpg - 1) / cpg;
  const dim3 gr(nrb, p->B * p->S, groups);
  prof_mark("fft_generic", p->stream, false);
  SENSE_LAUNCH_CLS(fft_class(p->fW), k_row_combine, gr, smem_rows_inv(p->W), p->stream, p->S, p->C, p->H, p->w.T,
                   p->maps, out, dev(p->fW), mode, xin, lam_host, lam_dev, groups > 1 ? cpg : p->C);
  if (groups > 1) {
    const int HW = p->H * p->W;
    const long long n = (long long)p->B * HW;
    const int grid = (int)std::min<long long>((n + 255) / 256, 2048LL);
    k_coil_groups_sum<<<grid, 256, 0, p->stream>>>(p->B, p->C, p->H, p->W, p->W, cpg, p->w.T, xin, lam_host,
                                                    lam_dev, out);
    count_launch(p, 1);
  }
  prof_mark("fft_generic", p->stream, true);
  count_launch(p, 1);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int launch_forward_generic(sense_plan p, const float2* x, float2* y) {
  const dim3 gr((p->H + kRows - 1) / kRows, p->B * p->C);
  prof_mark("fft_generic", p->stream, false);
  SENSE_LAUNCH_CLS(fft_class(p->fW), k_row_expand, gr, smem_rows(p->W), p->stream, p->B, p->S, p->C, p->H, x,
                   p->maps, y, dev(p->fW), 0);
  prof_mark("fft_generic", p->stream, true);
  const dim3 gc((p->W + kCols - 1) / kCols, p->B * p->C);
  prof_mark("fft_generic", p->stream, false);
  SENSE_LAUNCH_CLS(fft_class(p->fH), k_col, gc, smem_cols(p->H), p->stream, p->W, y, y, dev(p->fH), p->mask,
                   p->mask_is_lines, 0, nullptr, 0);
  prof_mark("fft_generic", p->stream, true);
  count_launch(p, 2);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int launch_adjoint_generic(sense_plan p, const float2* y, float2* x) {
  if (p->lines.ok && p->lines.ncols > 0) {
    // line mask: column transforms of the sampled columns only, then the fused pruned row pass
    const dim3 gc((p->lines.ncols + kCols - 1) / kCols, p->B * p->C);
    prof_mark("adjoint_lines", p->stream, false);
    SENSE_LAUNCH_CLS(fft_class(p->fH), k_col, gc, smem_cols(p->H), p->stream, p->W, y, p->w.T, dev(p->fH),
                     p->mask, p->mask_is_lines, 1, p->lines.cols, p->lines.ncols);
    prof_mark("adjoint_lines", p->stream, true);
    count_launch(p, 1);
    NormalLaunch L;
    L.mode = NM_ADJ; L.x = p->w.T; L.out = x;
    return launch_normal_lines(p, L);
  }
  const dim3 gc((p->W + kCols - 1) / kCols, p->B * p->C);
  prof_mark("fft_generic", p->stream, false);
  SENSE_LAUNCH_CLS(fft_class(p->fH), k_col, gc, smem_cols(p->H), p->stream, p->W, y, p->w.T, dev(p->fH),
                   p->mask, p->mask_is_lines, 1, nullptr, 0);
  prof_mark("fft_generic", p->stream, true);
  count_launch(p, 1);
  return launch_row_combine(p, x, 1, nullptr, 0.f, nullptr);
}

void launch_col_normal(sense_plan p) {
  if (use_col256(p)) {
    const dim3 gc((p->W + kC6 - 1) / kC6, (p->B * p->C + kCol256Images - 1) / kCol256Images);
    k_col256<<<gc, 32 * kC6, smem_col256(), p->stream>>>(p->B * p->C, p->W, p->w.T, p->twtab + kTwTab, p->mask2s,
                                                         p->mask_is_lines);
    return;
  }
  const dim3 gc((p->W + kCols - 1) / kCols, p->B * p->C);
  SENSE_LAUNCH_CLS(fft_class(p->fH), k_col, gc, smem_cols(p->H), p->stream, p->W, p->w.T, p->w.T, dev(p->fH),
                   p->mask2s, p->mask_is_lines, 2, nullptr, 0);
}

// Normal operator with the Bluestein row passes (use_blue): forward rows, the column
// pass, inverse rows with the coil sum in groups across grid.z (about 1024 CTAs).
int launch_normal_blue(sense_plan p, const float2* x, float2* out, float lam_host, const double* lam_dev) {
  const int nrb = (p->H + kRB - 1) / kRB;
  prof_mark("fft_generic", p->stream, false);
  k_blue_rows_fwd<<<dim3(nrb, p->B * p->C), 64 * kRB, smem_blue(), p->stream>>>(p->C, p->H, p->W, x, p->maps,
                                                                                 p->w.T, p->twtab, p->blue);
  launch_col_normal(p);
  int groups = (1024 + nrb * p->B - 1) / (nrb * p->B);
  groups = groups < 1 ? 1 : (groups > p->C ? p->C : groups);
  const int cpg = (p->C + groups - 1) / groups;
  groups = (p->C + cpg - 1) / cpg;
  k_blue_rows_inv<<<dim3(nrb, p->B, groups), 64 * kRB, smem_blue(), p->stream>>>(
      p->C, p->H, p->W, p->w.T, p->maps, out, p->twtab, p->blue, x, lam_host, lam_dev, groups > 1 ? cpg : p->C);
  if (groups > 1) {
    const long long n = (long long)p->B * p->H * p->W;
    const int grid = (int)std::min<long long>((n + 255) / 256, 2048LL);
    k_coil_groups_sum<<<grid, 256, 0, p->stream>>>(p->B, p->C, p->H, p->W, p->W, cpg, p->w.T, x, lam_host,
                                                    lam_dev, out);
    count_launch(p, 1);
  }
  prof_mark("fft_generic", p->stream, true);
  count_launch(p, 3);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

// Normal operator with the direct W = 8 P row passes: forward rows, the column pass, inverse rows
// with the coil sum in groups across grid.z (about 1024 CTAs).
int launch_normal_r8p(sense_plan p, const float2* x, float2* out, float lam_host, const double* lam_dev) {
  const int nrb = (p->H + kR8Rows - 1) / kR8Rows;
  int groups = (1024 + nrb * p->B - 1) / (nrb * p->B);
  groups = groups < 1 ? 1 : (groups > p->C ? p->C : groups);
  const int cpg = (p->C + groups - 1) / groups;
  groups = (p->C + cpg - 1) / cpg;
  prof_mark("fft_generic", p->stream, false);
  SENSE_R8P_SWITCH(p->r8p,
    k_r8p_fwd<kP><<<dim3(nrb, p->B * p->C), 32 * kR8Rows, smem_r8p<kP>(), p->stream>>>(p->C, p->H, x, p->maps,
                                                                                       p->w.T, p->fW.tw))
  launch_col_normal(p);
  SENSE_R8P_SWITCH(p->r8p,
    k_r8p_inv<kP><<<dim3(nrb, p->B, groups), 32 * kR8Rows, smem_r8p<kP>(), p->stream>>>(
        p->C, p->H, p->w.T, p->maps, out, p->fW.tw, x, lam_host, lam_dev, groups > 1 ? cpg : p->C))
  if (groups > 1) {
    const long long n = (long long)p->B * p->H * p->W;
    const int grid = (int)std::min<long long>((n + 255) / 256, 2048LL);
    k_coil_groups_sum<<<grid, 256, 0, p->stream>>>(p->B, p->C, p->H, p->W, p->W, cpg, p->w.T, x, lam_host,
                                                    lam_dev, out);
    count_launch(p, 1);
  }
  prof_mark("fft_generic", p->stream, true);
  count_launch(p, 3);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int launch_normal_generic(sense_plan p, const float2* x, float2* out, float lam_host,
                          const double* lam_dev) {
  if (p->toep) return launch_normal_toeplitz(p, x, out, lam_host, lam_dev, nullptr);
  if (p->r8p) return launch_normal_r8p(p, x, out, lam_host, lam_dev);
  if (p->blue) return launch_normal_blue(p, x, out, lam_host, lam_dev);
  const dim3 gr((p->H + kRows - 1) / kRows, p->B * p->C);
  prof_mark("fft_generic", p->stream, false);
  SENSE_LAUNCH_CLS(fft_class(p->fW), k_row_expand, gr, smem_rows(p->W), p->stream, p->B, p->S, p->C, p->H, x,
                   p->maps, p->w.T, dev(p->fW), 1);
  prof_mark("fft_generic", p->stream, true);
  prof_mark("fft_generic", p->stream, false);
  launch_col_normal(p);
  prof_mark("fft_generic", p->stream, true);
  count_launch(p, 2);
  return launch_row_combine(p, out, 2, x, lam_host, lam_dev);
}

// The register-resident passes serve a length-512 axis (their index digits are fixed): the
// column pass 2H = 512, the row passes 2W = 512.
bool use_cols512(sense_plan p) { return p->H == 256; }
bool use_rows512(sense_plan p) { return p->W == 256; }

int toeplitz_prepare(sense_plan p, const float2* psf) {
  const int H2 = 2 * p->H, W2 = 2 * p->W;
  if (kRows * W2 > kThreads * kMaxPer || kRows * p->W > kThreads * kMaxPer) return SENSE_EUNSUPPORTED;
  const int sr = smem_rows(W2), sc = smem_cols(H2);
  if (sr > 200 * 1024 || sc > 200 * 1024) return SENSE_EUNSUPPORTED;
  if (!SENSE_SET_SMEM(k_tp_rows_fwd, sr) || !SENSE_SET_SMEM(k_tp_rows_inv, smem_rows_inv(W2)) ||
      !SENSE_SET_SMEM(k_tp_psf_rows, sr) || !SENSE_SET_SMEM(k_tp_cols, sc) || !SENSE_SET_SMEM(k_tp_psf_cols, sc))
    return SENSE_ECUDA;
  if (use_cols512(p) && cudaFuncSetAttribute(k_tp_cols512, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem_cols512()) != cudaSuccess)
    return SENSE_ECUDA;
  if (use_cols512(p) || use_rows512(p))
    if (int e = twtab_prepare(p)) return e;
  if (use_rows512(p) && (cudaFuncSetAttribute(k_tp_rows_fwd512, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem_rows512()) != cudaSuccess ||
                         cudaFuncSetAttribute(k_tp_rows_inv512, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem_rows512()) != cudaSuccess))
    return SENSE_ECUDA;
  SENSE_LAUNCH_CLS(fft_class(p->fW2), k_tp_psf_rows, (H2 + kRows - 1) / kRows, sr, p->stream, H2, psf,
                   p->psf_hat, dev(p->fW2));
  SENSE_LAUNCH_CLS(fft_class(p->fH2), k_tp_psf_cols, (W2 + kCols - 1) / kCols, sc, p->stream, W2, p->psf_hat,
                   dev(p->fH2), (float)(1.0 / ((double)H2 * W2)));
  count_launch(p, 2);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

// The Toeplitz operator's inverse row pass can also form the rows of Re<x, out> (one coil
// group: the register-resident row passes with every coil of a row in one CTA).
static int toeplitz_groups(sense_plan p, bool rows512) {
  const int nrb = rows512 ? (p->H + kR5 - 1) / kR5 : (p->H + kRows - 1) / kRows;
  const int target = rows512 ? 1024 : 2048;
  int groups = (target + nrb * p->B - 1) / (nrb * p->B);
  groups = groups < 1 ? 1 : (groups > p->C ? p->C : groups);
  const int cpg = (p->C + groups - 1) / groups;
  return (p->C + cpg - 1) / cpg;
}
bool toeplitz_fused_dot(sense_plan p) {
  return p->toep && use_rows512(p) && toeplitz_groups(p, true) == 1;
}

int launch_normal_toeplitz(sense_plan p, const float2* x, float2* out, float lam_host, const double* lam_dev,
                           double* dpart) {
  if (dpart && !toeplitz_fused_dot(p)) return SENSE_EUNSUPPORTED;
  const int W2 = 2 * p->W;
  const bool rows512 = use_rows512(p);
  prof_mark("toeplitz", p->stream, false);
  if (rows512) {
    const dim3 gr((p->H + kR5 - 1) / kR5, p->B * p->C);
    k_tp_rows_fwd512<<<gr, 64 * kR5, smem_rows512(), p->stream>>>(p->C, p->H, x, p->maps, p->w.T, p->twtab);
  } else {
    const dim3 gr((p->H + kRows - 1) / kRows, p->B * p->C);
    SENSE_LAUNCH_CLS(fft_class(p->fW2), k_tp_rows_fwd, gr, smem_rows(W2), p->stream, p->C, p->H, p->W, x, p->maps,
                     p->w.T, dev(p->fW2));
  }
  if (use_cols512(p)) {
    const dim3 gc((W2 + kC5 - 1) / kC5, (p->B * p->C + kTpImages - 1) / kTpImages);
    k_tp_cols512<<<gc, 64 * kC5, smem_cols512(), p->stream>>>(p->B * p->C, W2, p->w.T, p->twtab, p->psf_hat);
  } else {
    const dim3 gc((W2 + kCols - 1) / kCols, p->B * p->C);
    SENSE_LAUNCH_CLS(fft_class(p->fH2), k_tp_cols, gc, smem_cols(2 * p->H), p->stream, p->H, W2, p->w.T,
                     dev(p->fH2), p->psf_hat);
  }
  // inverse rows and coil combine, the coils split into groups across grid.z (about 2048 CTAs
  // of 256 threads, or 1024 of 512 with the register-resident pass)
  const int nrb = rows512 ? (p->H + kR5 - 1) / kR5 : (p->H + kRows - 1) / kRows;
  const int groups = toeplitz_groups(p, rows512);
  const int cpg = (p->C + groups - 1) / groups;
  const dim3 gr2(nrb, p->B, groups);
  if (rows512) {
    k_tp_rows_inv512<<<gr2, 64 * kR5, smem_rows512(), p->stream>>>(p->C, p->H, p->w.T, p->maps, out, p->twtab, x,
                                                                    lam_host, lam_dev, groups > 1 ? cpg : p->C,
                                                                    groups > 1 ? nullptr : dpart);
  } else {
    SENSE_LAUNCH_CLS(fft_class(p->fW2), k_tp_rows_inv, gr2, smem_rows_inv(W2), p->stream, p->C, p->H, p->W, p->w.T,
                     p->maps, out, dev(p->fW2), x, lam_host, lam_dev, groups > 1 ? cpg : p->C);
  }
  if (groups > 1) {
    const long long n = (long long)p->B * p->H * p->W;
    const int grid = (int)std::min<long long>((n + 255) / 256, 2048LL);
    k_coil_groups_sum<<<grid, 256, 0, p->stream>>>(p->B, p->C, p->H, p->W, W2, cpg, p->w.T, x, lam_host, lam_dev,
                                                    out);
    count_launch(p, 1);
  }
  prof_mark("toeplitz", p->stream, true);
  count_launch(p, 3);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

extern "C" int sense_toeplitz_psf(const float* traj, int M, int H, int W, void* psf, void* stream) {
  if (M <= 0 || H <= 0 || W <= 0 || (H & 1) || (W & 1)) return SENSE_EINVAL_SHAPE;
  if (!traj || !psf || ((uintptr_t)traj & 7u) || ((uintptr_t)psf & 15u)) return SENSE_EINVAL_PTR;
  const dim3 g((2 * W + kPsfTile - 1) / kPsfTile, (2 * H + kPsfTile - 1) / kPsfTile);
  k_tp_psf<<<g, 256, 0, static_cast<cudaStream_t>(stream)>>>(M, H, W, traj, static_cast<float2*>(psf));
  prof_count(1);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}
