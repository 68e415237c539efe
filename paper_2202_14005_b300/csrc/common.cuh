// Shared device helpers of libsense: complex float2 arithmetic, register DFTs of
// small power-of-two length, status words and fixed-order reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sense.h"

#define SENSE_HD __host__ __device__ __forceinline__
#define SENSE_D __device__ __forceinline__

// ------------------------------------------------------------------ complex
SENSE_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
SENSE_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
SENSE_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
SENSE_HD float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
SENSE_HD float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// acc + a * b
SENSE_HD float2 cfma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
  return acc;
}
// acc + conj(a) * b
SENSE_HD float2 cfmac(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
  return acc;
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
SENSE_HD float2 cmul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(2 pi j / 32), j = 0..8 (the other angles follow by symmetry); literal
// values of the mathematical constants.
SENSE_D float cos32(int j) {
  return j == 0 ? 1.0f
       : j == 1 ? 0.98078528040323044913f
       : j == 2 ? 0.92387953251128675613f
       : j == 3 ? 0.83146961230254523708f
       : j == 4 ? 0.70710678118654752440f
       : j == 5 ? 0.55557023301960222474f
       : j == 6 ? 0.38268343236508977173f
       : j == 7 ? 0.19509032201612826785f
       : 0.0f;
}
// e^{-2 pi i k / n} (INV: e^{+2 pi i k / n}) for n | 32, 0 <= k < n.
template <bool INV>
SENSE_D float2 tw_pow2(int k, int n) {
  const int j = k * (32 / n);  // angle in units of 2 pi / 32
  const int q = j >> 3, r = j & 7;
  float c, s;                  // cos and sin of 2 pi j / 32
  if (q == 0) { c = cos32(r); s = cos32(8 - r); }
  else if (q == 1) { c = -cos32(8 - r); s = cos32(r); }
  else if (q == 2) { c = -cos32(r); s = -cos32(8 - r); }
  else { c = cos32(8 - r); s = -cos32(r); }
  return INV ? make_float2(c, s) : make_float2(c, -s);
}
// a * e^{-/+ 2 pi i k / n}; trivial angles are folded at compile time.
template <bool INV>
SENSE_D float2 cmul_tw(float2 a, int k, int n) {
  if (k == 0) return a;
  if (4 * k == n) return cmul_mi<INV>(a);
  if (2 * k == n) return make_float2(-a.x, -a.y);
  if (4 * k == 3 * n) return cmul_mi<!INV>(a);
  return cmul(a, tw_pow2<INV>(k, n));
}

constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
// Bit reversal of i within `bits` <= 5 bits, loop- and call-free so that it
// folds to a constant inside unrolled loops.
SENSE_HD int bitrev5(int i, int bits) {
  const int r = ((i & 1) << 4) | ((i & 2) << 2) | (i & 4) | ((i & 8) >> 2) | ((i & 16) >> 4);
  return r >> (5 - bits);
}

// In-register DFT of length N (power of two <= 32): v[k] <- sum_n v[n] w^{nk},
// w = e^{-2 pi i / N} (INV: e^{+2 pi i / N}), unnormalised.  Radix-2
// decimation in time; indices and twiddles resolve at compile time.
template <int N, bool INV>
SENSE_D void dft_pow2(float2 (&v)[N]) {
  constexpr int LB = ilog2c(N);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int j = bitrev5(i, LB);
    if (i < j) { const float2 t = v[i]; v[i] = v[j]; v[j] = t; }
  }
#pragma unroll
  for (int s = 0; s < LB; ++s) {
    const int half = 1 << s;
#pragma unroll
    for (int bf = 0; bf < N / 2; ++bf) {
      const int k = bf & (half - 1);
      const int i = ((bf >> s) << (s + 1)) + k;
      const float2 a = v[i];
      const float2 b = cmul_tw<INV>(v[i + half], k, 2 * half);
      v[i] = cadd(a, b);
      v[i + half] = csub(a, b);
    }
  }
}

// ------------------------------------------------ programmatic dependent launch
// Programmatic dependent launch (a kernel launched with programmatic stream serialisation may
// start while the kernel before it in the stream is still running): griddep_wait returns once
// that kernel has completed and its memory is visible (at once for a kernel launched without
// the attribute); griddep_release lets the next such kernel start its own prologue.  A kernel
// calls griddep_release only after griddep_wait, so whenever a prologue runs, every kernel
// before its predecessor has completed.
SENSE_D void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
SENSE_D void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic stream serialisation (for the kernels that call griddep_wait before
// reading what the previous kernel wrote and before writing anything).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}

// ------------------------------------------------------------ device status
#define SENSE_DEVST_CG_BREAKDOWN SENSE_STATUS_CG_BREAKDOWN
#define SENSE_DEVST_NONFINITE SENSE_STATUS_NONFINITE

SENSE_D void set_status(int* st, int bit) {
  if (st) atomicOr(st, bit);
}

// --------------------------------------------------------- fixed-order sums
// Lane sum of part[lane], part[lane + 32], ... part[< n] in index order.  The loads of eight
// consecutive strides are issued before they are added (one L2 round trip per eight terms
// instead of one per term); the order of the additions is unchanged.
SENSE_D double lane_strided_sum(const double* part, int n, int lane) {
  double s = 0.0;
  int i = lane;
  for (; i + 7 * 32 < n; i += 8 * 32) {
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __ldcg(part + i + 32 * k);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
  }
  for (; i < n; i += 32) s += __ldcg(part + i);
  return s;
}
// Lane part of a strided sum (elements lane, lane + 32, ...) with the loads of each group of
// eight issued together and each group added as a pairwise tree (FP64 additions take long to
// complete, so the dependent chain is kept short); groups are added in order.  Deterministic.
SENSE_D double tree8(const double* v) {
  return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
}
SENSE_D double lane_tree_sum(const double* p, int n, int lane) {
  double s = 0.0;
  int i = lane;
  for (; i + 7 * 32 < n; i += 8 * 32) {
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __ldcg(p + i + 32 * k);
    s = i == lane ? tree8(v) : s + tree8(v);
  }
  for (; i < n; i += 32) s += __ldcg(p + i);
  return s;
}
// Two lane_tree_sum()s over arrays of the same length, loads issued together.
SENSE_D void lane_tree_sum2(const double* p0, const double* p1, int n, int lane, double& s0, double& s1) {
  s0 = 0.0;
  s1 = 0.0;
  int i = lane;
  for (; i + 7 * 32 < n; i += 8 * 32) {
    double v0[8], v1[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v0[k] = __ldcg(p0 + i + 32 * k);
      v1[k] = __ldcg(p1 + i + 32 * k);
    }
    s0 = i == lane ? tree8(v0) : s0 + tree8(v0);
    s1 = i == lane ? tree8(v1) : s1 + tree8(v1);
  }
  for (; i < n; i += 32) {
    s0 += __ldcg(p0 + i);
    s1 += __ldcg(p1 + i);
  }
}
// Warp sum in a fixed butterfly order (deterministic).
SENSE_D double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
SENSE_D float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------ compensated FP32 sums (float-float)
// A value carried as the unevaluated sum hi + lo of two floats.  Addition: Knuth's TwoSum
// recovers the rounding error of hi_a + hi_b exactly, the low parts are added to it, and
// Dekker's fast two-sum renormalises (|lo| <= ulp(hi) / 2): about 44 significant bits, on the
// FP32 pipes.  This GPU's FP64 units take tens of cycles per warp instruction, so sums that
// need more than FP32 accuracy are carried this way and converted to FP64 once.  The operation
// is symmetric in its operands (the TwoSum error is exact), so butterfly partners agree bitwise.
// Only additions and subtractions: nothing for the compiler to contract into an FMA.
SENSE_HD float2 ff_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bb = s - a.x;
  float e = (a.x - (s - bb)) + (b.x - bb);
  e += a.y + b.y;
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}
SENSE_HD double ff_to_d(float2 a) { return (double)a.x + (double)a.y; }
// Warp sum in a fixed butterfly order (deterministic, every lane gets the same value).
SENSE_D float2 warp_sum_ff(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float2 w;
    w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
    w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
    v = ff_add(v, w);
  }
  return v;
}
SENSE_D float2 warp_sum_ff(float v) { return warp_sum_ff(make_float2(v, 0.f)); }
// Lane part of a strided float-float sum (elements lane, lane + 32, ...): groups of eight loaded
// together and added as a pairwise tree, groups added in order (as lane_tree_sum).
SENSE_D float2 ff_tree8(const float2* v) {
  return ff_add(ff_add(ff_add(v[0], v[1]), ff_add(v[2], v[3])), ff_add(ff_add(v[4], v[5]), ff_add(v[6], v[7])));
}
SENSE_D float2 lane_tree_sum_ff(const float2* p, int n, int lane) {
  float2 s = make_float2(0.f, 0.f);
  int i = lane;
  for (; i + 7 * 32 < n; i += 8 * 32) {
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __ldcg(p + i + 32 * k);
    s = i == lane ? ff_tree8(v) : ff_add(s, ff_tree8(v));
  }
  for (; i < n; i += 32) s = ff_add(s, __ldcg(p + i));
  return s;
}
