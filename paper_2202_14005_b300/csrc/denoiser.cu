// MoDL residual CNN denoiser D_W(x) = x + CNN(x) (Sec. 2.3.2, Eq. 6), forward
// and reverse mode.  CNN: 3x3 convolutions 2 -> 64 -> 64 -> 64 -> 64 -> 2 with
// biases and ReLU between them; the complex image enters as two real channels.
//
// Activations are BF16, channels-last [B][H][W][64]; accumulation is FP32.
// * Layers with a 64-channel input (the 64 -> 64 layers, forward and input
//   gradient; the 64 -> 2 last layer and the first layer's input gradient):
//   implicit GEMM on the 5th-gen tensor cores (k_conv64).  One MMA tile is 128
//   consecutive pixels of one image row (M = 128); K = 9 taps x 64 channels.  A
//   TMA tensor copy brings the 3 x 130-pixel halo into shared memory with the
//   128-byte swizzle, so each tap is the same K-major operand at a shifted
//   start address; weights sit in shared memory K-major; the FP32 accumulator
//   lives in tensor memory (two buffers, so the epilogue of one tile overlaps
//   the MMAs of the next).  N = 64 for the 64 -> 64 layers (epilogue: bias +
//   ReLU, or the ReLU mask of the layer input, rounded to BF16); N = 16 with the
//   three horizontal taps on the output side for the 64 -> 2 layers.
// * Weight gradients of the 64 -> 64 layers: a contraction over pixels on the
//   tensor cores (k_wgrad64, accumulators in tensor memory).
// * The 2 -> 64 first layer and the last layer's input gradient: warp-level
//   tensor cores (mma.sync, k_2to64); the weight gradients of the two
//   2-channel layers: CUDA cores (k_wgrad_l1, k_wgrad_l5).  Every weight
//   gradient is a set of per-chunk FP32 partials reduced in a fixed order
//   (deterministic) and added to the caller's FP32 buffer.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "plan.cuh"
#include "tc.cuh"

namespace {

constexpr int CH = 64;
// Convolutions with a 64-channel input run as implicit GEMMs on tcgen05 (M = 128 halo pixels of
// one image row, K = 16 channels per MMA), in one of two forms:
//  * NOUT = 64 (the 64 -> 64 layers): 36 MMAs per tile, one per (tap, 16-channel step), the tap's
//    pixel offset dx applied as a 128-byte start offset of the A operand; N = 64; 128 outputs
//    per tile from a 130-pixel halo.
//  * NOUT = 16 (the 64 -> 2 layers): the horizontal tap moved to the output side: 12 MMAs, one per
//    (dy, 16-channel step), with the three taps' weights stacked along N (column 2 dx + c), and the
//    epilogue adds D_0[q] + D_1[q + 1] + D_2[q + 2] across lanes; 126 outputs per tile from a
//    128-pixel halo.  (For N = 64 the cross-lane epilogue costs more than the MMAs it saves.)
constexpr int TILE_M = 128;                   // MMA M
constexpr int CONV_THREADS = 160;             // warps 0-3 epilogue (one TMEM lane quadrant each), warp 4 producer
constexpr int NHALO = 3;                      // halo slots (TMA runs two tiles ahead of the MMAs)
constexpr int NBARS = 1 + 2 * NHALO + 2 + 2;  // weights, halo full/empty, TMEM full/empty
// Shared-memory layout and tile geometry per NOUT: packed weights, NHALO halo slots (1 KB
// aligned), bias, the epilogue warps' boundary exchange (NOUT = 16), barriers.
template <int NOUT>
struct ConvLayout {
  static constexpr bool SHIFT = NOUT == 16;             // output-side horizontal tap
  static constexpr int CO = NOUT == 64 ? 64 : 2;        // output channels
  static constexpr int NCOL = NOUT;                     // MMA N
  static constexpr int HALO_PX = SHIFT ? TILE_M : TILE_M + 2;
  static constexpr int TILE_OUT = SHIFT ? TILE_M - 2 : TILE_M;
  static constexpr int HALO_ROWB = HALO_PX * 64 * 2;
  static constexpr int HALO_TX = 3 * HALO_ROWB;
  static constexpr int HALO_SLOT = (HALO_TX + 1023) & ~1023;
  static constexpr int WP = (SHIFT ? 3 : 9) * 8 * NCOL * 16;  // [dy][g][n][8] or [tap][g][n][8]
  static constexpr int OFF_W = 0;
  static constexpr int OFF_H0 = (WP + 1023) & ~1023;
  static constexpr int OFF_BIAS = OFF_H0 + NHALO * HALO_SLOT;
  static constexpr int OFF_XCH = OFF_BIAS + 64 * 4;     // [2 tiles][4 warps][4 rows][CO] floats
  static constexpr int OFF_BAR = OFF_XCH + (SHIFT ? 2 * 4 * 4 * CO * 4 : 0);
  static constexpr int SMEM = OFF_BAR + NBARS * 8 + 16 + 1024;  // + slack to realign the base to 1 KB
  static constexpr int TCOL = NOUT;                     // TMEM columns between the two accumulators
  static constexpr int TMEM_COLS = 2 * NOUT < 32 ? 32 : 2 * NOUT;
};
constexpr int WPACK_BYTES = ConvLayout<64>::WP;  // 73728 (bf16 [tap][g][64][8])
constexpr int WP16_BYTES = ConvLayout<16>::WP;   // 6144 (64 -> 2 tables [dy][g][16][8])

// Offsets (floats) into the flat MoDL weight vector: w_l [Cout][Cin][3][3], b_l [Cout].
struct ModlOffsets {
  int w[5], b[5], total;
};
constexpr int kChans[6] = {2, 64, 64, 64, 64, 2};
ModlOffsets modl_offsets() {
  ModlOffsets o;
  int p = 0;
  for (int l = 0; l < 5; ++l) {
    o.w[l] = p;
    p += kChans[l] * kChans[l + 1] * 9;
    o.b[l] = p;
    p += kChans[l + 1];
  }
  o.total = p;
  return o;
}

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const uint32_t d = smem_u32(dst);
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }


// ------------------------------------------------------------ weight packing
// Convolution weights into K-major operand layouts (bf16), one launch for all eight tables:
//  blockIdx.y = 2 * layer + dgrad, the 64 -> 64 layers, [tap][g][n][8]:
//   forward:        n = cout, k-chunk g over cin:  W[n][g*8+e][tap]
//   input gradient: n = cin,  k-chunk g over cout: W[g*8+e][n][8 - tap] (flipped taps)
//  blockIdx.y = 6 (last layer forward) and 7 (first-layer input gradient), [dy][g][16][8] with
//  row n = 2 dx + c (c < 2) holding tap (dy, dx), output channel c; rows 6..15 zero.
struct PackArgs {
  const float* w[3];
  __nv_bfloat16* fwd[3];
  __nv_bfloat16* dgr[3];
  const float* w1;       // first layer [64][2][9]
  const float* w5;       // last layer [2][64][9]
  __nv_bfloat16* t5;     // last layer forward: w5[c][g*8+e][3 dy + dx] at n = 2 dx + c
  __nv_bfloat16* t1;     // first layer input gradient: w1[g*8+e][c][8 - (3 dy + dx)] at n = 2 dx + c
  uint32_t* f1;          // first layer forward, mma.sync B fragments [2 ks][8 nt][32 lanes][2]
  uint32_t* f5;          // last layer input gradient, B fragments [4 ks][8 nt][32 lanes][2]
};
// mma.sync m16n8k16 B fragment element pair (k, k + 1) of column j for the 2 -> 64 layers:
//   first layer forward: k = 9 c + tap < 18, W = w1[j][c][tap]
//   last layer input gradient: k = 18 part + 9 c + tap < 54, W = w5[c][j][tap] (each BF16 term)
__device__ __forceinline__ float w2to64(const float* w, int mode, int k, int j) {
  if (k >= (mode == 0 ? 18 : 54)) return 0.f;
  const int kk = k % 18, c = kk / 9, tap = kk % 9;
  return mode == 0 ? w[(j * 2 + c) * 9 + tap] : w[(c * CH + j) * 9 + tap];
}
__global__ void k_pack64(const PackArgs a) {
  griddep_wait();  // launched with programmatic serialisation: nothing is read before this
  griddep_release();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 9*8*64*8
  if (blockIdx.y >= 8) {  // B fragments of the 2 -> 64 layers, in the order a lane loads them
    const int mode = blockIdx.y - 8, ks_n = mode == 0 ? 2 : 4;
    if (i >= ks_n * 8 * 32 * 2) return;
    const int hf = i & 1, lane = (i >> 1) & 31, nt = (i >> 6) & 7, ks = i >> 9;
    const int gid = lane >> 2, tig = lane & 3;
    const int k = 16 * ks + 2 * tig + 8 * hf, j = 8 * nt + gid;
    const float* w = mode == 0 ? a.w1 : a.w5;
    __nv_bfloat162 v = __floats2bfloat162_rn(w2to64(w, mode, k, j), w2to64(w, mode, k + 1, j));
    (mode == 0 ? a.f1 : a.f5)[i] = *reinterpret_cast<uint32_t*>(&v);
    return;
  }
  if (blockIdx.y >= 6) {  // 64 -> 2 tables of the first and last layers (N = 16, 6 live rows)
    if (i >= 3 * 8 * 16 * 8) return;
    const int e = i & 7, n = (i >> 3) & 15, g = (i >> 7) & 7, dy = i >> 10;
    float v = 0.f;
    if (n < 6) {
      const int dx = n >> 1, c = n & 1, tap = dy * 3 + dx;
      v = (blockIdx.y == 6) ? a.w5[(c * CH + g * 8 + e) * 9 + tap] : a.w1[((g * 8 + e) * 2 + c) * 9 + (8 - tap)];
    }
    (blockIdx.y == 6 ? a.t5 : a.t1)[i] = __float2bfloat16_rn(v);
    return;
  }
  if (i >= 9 * 8 * CH * 8) return;
  const int l = blockIdx.y >> 1, dgrad = blockIdx.y & 1;
  const float* w = a.w[l];
  const int e = i & 7, n = (i >> 3) & 63, g = (i >> 9) & 7, tap = i >> 12;
  const float v = !dgrad ? w[(n * CH + g * 8 + e) * 9 + tap] : w[((g * 8 + e) * CH + n) * 9 + (8 - tap)];
  (dgrad ? a.dgr[l] : a.fwd[l])[i] = __float2bfloat16_rn(v);
}

// ------------------------------------------------------- tcgen05 convolution
struct ConvArgs {
  int B, H, W, ntw;
  const __nv_bfloat16* wpack;
  const float* bias;            // forward: [64]
  const __nv_bfloat16* aprev;   // input gradient: ReLU mask source [B][H][W][64]
  __nv_bfloat16* out;           // [B][H][W][64]
  int mode;                     // 0 forward, 1 input gradient (64 -> 64); 2 last layer, 3 first-layer input gradient (64 -> 2)
  const float2* res;            // modes 2/3: residual added to the two output channels
  float2* out2;                 // modes 2/3: complex output [B][H][W]
  int* status;
};

__device__ __forceinline__ void tile_coords(int t, int H, int ntw, int& b, int& h, int& wt) {
  wt = t % ntw;
  const int r = t / ntw;
  h = r % H;
  b = r / H;
}

template <int NOUT>
__device__ __forceinline__ void issue_halo(const CUtensorMap* map, uint8_t* dst, uint64_t* bar, int t,
                                           int H, int ntw) {
  using CL = ConvLayout<NOUT>;
  int b, h, wt;
  tile_coords(t, H, ntw, b, h, wt);
  mbar_expect_tx(bar, CL::HALO_TX);
  // one box {64 channels, HALO_PX pixels, 3 rows}: [row][pixel][128 bytes], 128-byte swizzled;
  // halo pixel p is image pixel wt * TILE_OUT - 1 + p
  tma_load_4d(dst, map, 0, wt * CL::TILE_OUT - 1, h - 1, b, bar);
}

template <int NOUT>
__device__ __forceinline__ void issue_mma(uint32_t tmem_d, uint32_t halo, uint32_t wts) {
  using CL = ConvLayout<NOUT>;
  constexpr int NCOL = CL::NCOL;
  const uint32_t idesc = umma_idesc_bf16(TILE_M, NCOL);
  if constexpr (CL::SHIFT) {
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        // A: the 128 halo pixels of row dy, channels 16 kk .. 16 kk + 15; B: taps (dy, 0..2)
        const uint64_t ad = umma_desc_sw128(halo + dy * CL::HALO_ROWB + kk * 32);
        const uint64_t bd = umma_desc(wts + (dy * 8 + 2 * kk) * (NCOL * 16), NCOL * 16, 128);
        umma_bf16(tmem_d, ad, bd, idesc, (dy | kk) != 0);
      }
    }
  } else {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3, dx = tap - dy * 3;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        // A: 128 pixels starting at halo pixel (dy, dx), channels 16 kk .. 16 kk + 15
        const uint64_t ad = umma_desc_sw128(halo + (dy * CL::HALO_PX + dx) * 128 + kk * 32);
        const uint64_t bd = umma_desc(wts + (tap * 8 + 2 * kk) * (NCOL * 16), NCOL * 16, 128);
        umma_bf16(tmem_d, ad, bd, idesc, (tap | kk) != 0);
      }
    }
  }
}

// Epilogue helpers: 16 output channels of one pixel, bias + ReLU (forward) or the ReLU mask of
// the previous activation (input gradient), stored as BF16.
__device__ __forceinline__ void conv_store16(const float (&o)[16], int cb, int mode, const float* s_bias,
                                             const uint4 (&mrow)[8], __nv_bfloat16* dst) {
  float v[16];
  if (mode == 0) {
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = fmaxf(o[e] + s_bias[cb * 16 + e], 0.f);
  } else {
    const uint4 m0 = mrow[2 * cb], m1 = mrow[2 * cb + 1];
    const __nv_bfloat16* mb0 = reinterpret_cast<const __nv_bfloat16*>(&m0);
    const __nv_bfloat16* mb1 = reinterpret_cast<const __nv_bfloat16*>(&m1);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      v[e] = (bf(mb0[e]) > 0.f) ? o[e] : 0.f;
      v[8 + e] = (bf(mb1[e]) > 0.f) ? o[8 + e] : 0.f;
    }
  }
  uint4 o0, o1;
  __nv_bfloat162* p0 = reinterpret_cast<__nv_bfloat162*>(&o0);
  __nv_bfloat162* p1 = reinterpret_cast<__nv_bfloat162*>(&o1);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    p0[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    p1[e] = __floats2bfloat162_rn(v[8 + 2 * e], v[8 + 2 * e + 1]);
  }
  uint4* op = reinterpret_cast<uint4*>(dst + cb * 16);
  op[0] = o0;
  op[1] = o1;
}

// Named barrier of the four epilogue warps (the producer warp does not take part).
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Warp-specialised persistent kernel, one 128-pixel row segment per tile, 3x3 taps as 36 MMAs of
// K = 16 over the halo (M = 128 pixels, N = NOUT).  NOUT = 64: the 64 -> 64 layers (epilogue
// bias + ReLU, or the input gradient masked by the previous activation).  NOUT = 16: the 64 -> 2
// layers with two live columns (mode 2, last layer: out = x + b5 + acc; mode 3, first-layer
// input gradient with flipped taps: gx = gout + acc).  Warp 4 (one lane) is the producer: it streams tile halos
// into NHALO shared slots with TMA and issues each tile's 36 MMAs into one of two TMEM halves as
// soon as the halo has landed and the epilogue has drained that half.  Warps 0-3 run the epilogue
// of every tile (warp w reads TMEM lanes 32w..32w+31: pixels 32w..32w+31).  Hand-offs go through
// mbarriers only:
//   halo_full[s]  TMA of slot s landed            (expect-tx, producer waits)
//   halo_empty[s] MMAs reading slot s finished    (tcgen05.commit, producer waits before reuse)
//   tm_full[t]    MMAs into TMEM half t finished  (tcgen05.commit, epilogue waits)
//   tm_empty[t]   four epilogue warps drained t   (count 4, producer waits before reuse)
// Tile j uses slot j % NHALO (use index j / NHALO) and TMEM half j % 2 (use index j / 2); the
// parity waited for is that use index's low bit.  Every wait is bounded: a role that gives up
// records an error, and the CTA waits (bounded) for whatever it still has in flight, frees its
// tensor memory and returns with SENSE_STATUS_DEVICE_TIMEOUT set.
template <int NOUT>
__global__ void __launch_bounds__(CONV_THREADS, 1)
k_conv64(const __grid_constant__ CUtensorMap tmap, const ConvArgs a) {
  using CL = ConvLayout<NOUT>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  uint8_t* s_halo = smem + CL::OFF_H0;
  float* s_bias = reinterpret_cast<float*>(smem + CL::OFF_BIAS);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + CL::OFF_BAR);
  uint64_t* w_full = bars;
  uint64_t* halo_full = bars + 1;
  uint64_t* halo_empty = bars + 1 + NHALO;
  uint64_t* tm_full = bars + 1 + 2 * NHALO;
  uint64_t* tm_empty = bars + 3 + 2 * NHALO;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + NBARS);
  int* s_err = reinterpret_cast<int*>(s_tmem + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = a.B * a.H * a.ntw;
  const int n = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (tid == 0) {
    mbar_init(w_full, 1);
    for (int k = 0; k < NHALO; ++k) {
      mbar_init(&halo_full[k], 1);
      mbar_init(&halo_empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&tm_full[k], 1);
      mbar_init(&tm_empty[k], 4);
    }
    *s_err = 0;
    fence_mbar_init();
  }
  if (tid < CH) s_bias[tid] = (a.mode == 0 || (a.mode == 2 && tid < 2)) ? a.bias[tid] : 0.f;
  if (warp == 0) {
    tmem_alloc(s_tmem, CL::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  // The packed weights (and the bias above) come from launches at least two kernels back, so they
  // load before the wait for the previous kernel; the halos, masks and residuals it may have
  // written, and every store, come after.
  if (warp == 4 && lane == 0 && n > 0) {
    mbar_expect_tx(w_full, CL::WP);
    bulk_load(smem + CL::OFF_W, a.wpack, CL::WP, w_full);
  }
  griddep_wait();
  griddep_release();

  // producer bookkeeping (lane 0 of warp 4): what it issued and what it has seen complete
  int tma_issued = 0, mma_issued = 0;
  if (warp == 4) {
    if (lane == 0 && n > 0) {
      const uint32_t sw = smem_u32(smem + CL::OFF_W);
      bool ok = true;
      const int pre = n < 2 ? n : 2;
      for (int j = 0; j < pre; ++j) {
        issue_halo<NOUT>(&tmap, s_halo + j * CL::HALO_SLOT, &halo_full[j], blockIdx.x + j * gridDim.x, a.H, a.ntw);
        ++tma_issued;
      }
      ok = mbar_wait(w_full, 0);
      for (int i = 0; i < n && ok; ++i) {
        const int s = i % NHALO, t = i & 1;
        ok = mbar_wait(&halo_full[s], (i / NHALO) & 1);
        if (ok && i >= 2) ok = mbar_wait(&tm_empty[t], ((i - 2) >> 1) & 1);
        if (!ok) break;
        tc_fence_after();
        issue_mma<NOUT>(tmem + t * CL::TCOL, smem_u32(s_halo + s * CL::HALO_SLOT), sw);
        umma_commit(&tm_full[t]);
        umma_commit(&halo_empty[s]);
        ++mma_issued;
        // refill the slot of tile i - 1 with tile i + 2 once the MMAs of tile i - 1 are done
        if (i + 2 < n) {
          const int s2 = (i + 2) % NHALO;
          if (i >= 1) ok = mbar_wait(&halo_empty[s2], ((i - 1) / NHALO) & 1);
          if (!ok) break;
          issue_halo<NOUT>(&tmap, s_halo + s2 * CL::HALO_SLOT, &halo_full[s2], blockIdx.x + (i + 2) * gridDim.x,
                           a.H, a.ntw);
          ++tma_issued;
        }
      }
      if (!ok) atomicExch(s_err, 1);
    }
  } else if constexpr (!CL::SHIFT) {
    // epilogue (NOUT = 64): warp w owns pixels 32w .. 32w + 31 of each tile
    for (int i = 0; i < n; ++i) {
      const int t = i & 1;
      int b, h, wt;
      tile_coords(blockIdx.x + i * gridDim.x, a.H, a.ntw, b, h, wt);
      const int px = wt * CL::TILE_OUT + warp * 32 + lane;
      const bool valid = px < a.W;
      const size_t pix = ((size_t)b * a.H + h) * a.W + px;
      // input-gradient mode: the whole 128-byte ReLU-mask row of this pixel in one batch of loads,
      // issued before the wait for the tile's accumulators
      uint4 mrow[8];
      if (a.mode == 1 && valid) {
        const uint4* ap = reinterpret_cast<const uint4*>(a.aprev + pix * CH);
#pragma unroll
        for (int q = 0; q < 8; ++q) mrow[q] = ap[q];
      }
      if (!mbar_wait(&tm_full[t], (i >> 1) & 1)) {
        atomicExch(s_err, 1);
        break;
      }
      tc_fence_after();
      float acc[64];
      tmem_ld64(tmem + ((uint32_t)(warp * 32) << 16) + t * CL::TCOL, acc);
      // the accumulators are in registers: hand the TMEM half back to the producer
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tm_empty[t]);
      if (valid) {
#pragma unroll
        for (int cb = 0; cb < 4; ++cb) {
          float o[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) o[e] = acc[cb * 16 + e];
          conv_store16(o, cb, a.mode, s_bias, mrow, a.out + pix * CH);
        }
      }
    }
  } else {
    // epilogue (NOUT = 16, 64 -> 2): warp w owns halo pixels 32w .. 32w + 31 of each tile (TMEM
    // lanes).  Lane l forms the output at halo pixel p = 32w + l from D_0[p] + D_1[p + 1] +
    // D_2[p + 2]: neighbours in the warp by shuffles; lanes 30 and 31 need lanes 0 and 1 of the
    // next warp, which publish D_1[p0] + D_2[p0 + 1] (for lane 31) and D_2[p0] (for lane 30) in the
    // exchange buffer while lanes 30 and 31 park their partial sums there; after one named barrier
    // of the epilogue warps they finish.  After a timed-out wait a warp stops waiting and reading
    // TMEM but keeps taking part in the barriers (one per tile).
    constexpr int CO = CL::CO;
    float* xch_base = reinterpret_cast<float*>(smem + CL::OFF_XCH);
    bool fail = false;
    for (int i = 0; i < n; ++i) {
      const int t = i & 1;
      int b, h, wt;
      tile_coords(blockIdx.x + i * gridDim.x, a.H, a.ntw, b, h, wt);
      const int p = warp * 32 + lane;
      const int px = wt * CL::TILE_OUT + p;
      const bool valid = p < CL::TILE_OUT && px < a.W;
      const size_t pix = ((size_t)b * a.H + h) * a.W + px;
      // the residual term of this pixel, loaded before the wait for the tile's accumulators
      const float2 rv = valid ? a.res[pix] : make_float2(0.f, 0.f);
      if (!fail) {
        const bool ok_wait = mbar_wait(&tm_full[t], (i >> 1) & 1);
        if (!ok_wait && lane == 0) atomicExch(s_err, 1);
        fail = __any_sync(0xffffffffu, !ok_wait);
      }
      tc_fence_after();
      float* xw = xch_base + (size_t)(t * 4 + warp) * 4 * CO;             // this warp's rows
      const float* xn = xch_base + (size_t)(t * 4 + warp + 1) * 4 * CO;   // the next warp's rows
      const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16) + t * CL::TCOL;
      float d[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (!fail) tmem_ld8(trow, d);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tm_empty[t]);
      float o[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float s1 = __shfl_down_sync(0xffffffffu, d[2 + c], 1);
        const float s2 = __shfl_down_sync(0xffffffffu, d[4 + c], 2);
        const float s21 = __shfl_down_sync(0xffffffffu, d[4 + c], 1);
        o[c] = d[c] + (lane < 31 ? s1 : 0.f) + (lane < 30 ? s2 : 0.f);
        if (lane == 0) {
          xw[0 * CO + c] = d[2 + c] + s21;  // D_1[p0] + D_2[p0 + 1]
          xw[1 * CO + c] = d[4 + c];        // D_2[p0]
        }
        if (lane >= 30) xw[(2 + lane - 30) * CO + c] = o[c];
      }
      if (lane < 30 && valid) a.out2[pix] = make_float2(rv.x + s_bias[0] + o[0], rv.y + s_bias[1] + o[1]);
      epi_bar();
      if (lane >= 30 && warp < 3 && valid) {
        const float* part = xw + (2 + lane - 30) * CO;
        const float* add = xn + (lane == 31 ? 0 : 1) * CO;
        a.out2[pix] = make_float2(rv.x + s_bias[0] + (part[0] + add[0]), rv.y + s_bias[1] + (part[1] + add[1]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*s_err && tid == 4 * 32) {
    set_status(a.status, SENSE_STATUS_DEVICE_TIMEOUT);
    // bounded drain of everything still in flight before shared and tensor memory are released:
    // every issued halo copy, and the last committed MMA batch (commits cover all earlier MMAs)
    for (int j = tma_issued > NHALO ? tma_issued - NHALO : 0; j < tma_issued; ++j)  // latest use of each slot
      mbar_wait(&halo_full[j % NHALO], (j / NHALO) & 1, 1u << 20);
    if (mma_issued > 0) {
      const int j = mma_issued - 1;
      mbar_wait(&halo_empty[j % NHALO], (j / NHALO) & 1, 1u << 20);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, CL::TMEM_COLS);
}

// ------------------------------------------------ 2-channel layers
// All convolution weights are used in BF16 (rounded when packed); sums are FP32.

// 2 -> 64 on the warp-level tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation).
// A CTA takes k2Rows image rows of one slice and stages their 2-channel (k2Rows + 2) x (W + 2)
// neighbourhood (zero outside the image); each warp takes 16-pixel groups of a row:
//   out[p][j] = sum_k A[p][k] W[k][j],  A = im2col of the neighbourhood, W in BF16,
//   mode 0 (first layer):   k = 9 c + tap (18, padded to 32), A = BF16(x) at (dy, dx); the
//                           products are exact, so only the summation order differs from a
//                           sequential FP32 sum; out = relu(b + sum)
//   mode 1 (last layer input gradient): k = 18 part + 9 c + tap (54, padded to 64), A = the FP32
//                           gradient at (2 - dy, 2 - dx) as three BF16 terms g1 + g2 + g3 (24
//                           significant bits); out = [a4 > 0] * sum, W = w5[c][j][tap]
// The 16 x 64 result of a group goes through shared memory (rows padded to 144 bytes) so that
// pixels are written as whole 128-byte rows, the ReLU mask of mode 1 read the same way.
constexpr int k2Rows = 2;
constexpr int k2Threads = 256;
constexpr int k2Ld = 72;  // bf16 per staged output row (144 bytes: conflict-free fragment stores)
int k2_smem(int W) {
  return (k2Rows + 2) * (W + 2) * (int)sizeof(float2) + (k2Threads / 32) * 16 * k2Ld * 2 + 4 * 8 * 32 * 2 * 4;
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

template <int MODE>
__global__ void __launch_bounds__(k2Threads) k_2to64(int B, int H, int W, const float2* src, const uint32_t* frag,
                                                     const float* bias, const __nv_bfloat16* mask_src,
                                                     __nv_bfloat16* out) {
  constexpr int KS = MODE == 0 ? 2 : 4;  // k-steps of 16
  constexpr int KV = MODE == 0 ? 18 : 54;
  griddep_wait();  // launched with programmatic serialisation: the fragments and the input come
  griddep_release();  // from the kernels before it
  extern __shared__ __align__(16) uint8_t dsm[];
  float2* s_n = reinterpret_cast<float2*>(dsm);  // [k2Rows + 2][W + 2]
  const int ld = W + 2;
  __nv_bfloat16* s_o = reinterpret_cast<__nv_bfloat16*>(dsm + (size_t)(k2Rows + 2) * ld * sizeof(float2));
  uint2* s_f = reinterpret_cast<uint2*>(s_o + (k2Threads / 32) * 16 * k2Ld);  // [KS][8][32] fragment pairs
  for (int i = threadIdx.x; i < KS * 8 * 32; i += blockDim.x) s_f[i] = reinterpret_cast<const uint2*>(frag)[i];
  const int nrb = (H + k2Rows - 1) / k2Rows;
  const int b = blockIdx.x / nrb, h0 = (blockIdx.x % nrb) * k2Rows;
  const int nrows = min(k2Rows, H - h0);
  for (int i = threadIdx.x; i < (nrows + 2) * ld; i += blockDim.x) {
    const int r = i / ld, q = i - r * ld;
    const int yy = h0 - 1 + r, xx = q - 1;
    float2 v = make_float2(0.f, 0.f);
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = src[((size_t)b * H + yy) * W + xx];
    if (MODE == 0) v = make_float2(bf(__float2bfloat16_rn(v.x)), bf(__float2bfloat16_rn(v.y)));
    s_n[i] = v;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tig = lane & 3;
  // B fragments (k-step ks, n-tile nt: b0 = W[16 ks + 2 tig (+1)][8 nt + gid], b1 = rows + 8) come
  // from the table packed with the weights, one shared-memory pair per (ks, nt) and lane
  // this lane's A columns: for k-step ks and slot sl (k = 16 ks + 2 tig + (sl & 1) + 8 (sl >> 1)),
  // the neighbourhood offset, channel and BF16 term (or -1 for padding)
  int aoff[KS][4], acomp[KS][4];
#pragma unroll
  for (int ks = 0; ks < KS; ++ks)
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
      const int k = 16 * ks + 2 * tig + (sl & 1) + 8 * (sl >> 1);
      if (k >= KV) {
        aoff[ks][sl] = 0;
        acomp[ks][sl] = -1;
      } else {
        const int part = k / 18, kk = k % 18, c = kk / 9, tap = kk % 9, dy = tap / 3, dx = tap % 3;
        aoff[ks][sl] = (MODE == 0) ? dy * ld + dx : (2 - dy) * ld + (2 - dx);
        acomp[ks][sl] = part * 2 + c;
      }
    }
  float bj[8][2];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) bj[nt][e] = (MODE == 0) ? bias[8 * nt + 2 * tig + e] : 0.f;
  __syncthreads();
  __nv_bfloat16* so = s_o + warp * 16 * k2Ld;
  const int ngw = (W + 15) / 16;  // groups per row
  for (int gi = warp; gi < nrows * ngw; gi += k2Threads / 32) {
    const int r = gi / ngw, w0 = (gi - r * ngw) * 16;
    const size_t prow = ((size_t)b * H + h0 + r) * W;
    // mode 1: this lane's four 16-byte chunks of the ReLU mask rows, loaded before the MMAs
    uint4 mk[4];
    if (MODE == 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = q * 32 + lane, px = w0 + (idx >> 3);
        mk[q] = px < W ? reinterpret_cast<const uint4*>(mask_src + (prow + px) * CH)[idx & 7]
                       : make_uint4(0u, 0u, 0u, 0u);
      }
    }
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      acc[nt][0] = acc[nt][2] = bj[nt][0];
      acc[nt][1] = acc[nt][3] = bj[nt][1];
    }
    const int pa = w0 + gid, pb = pa + 8;  // this lane's two pixels
    const float2* base_a = s_n + r * ld + pa;
    const float2* base_b = s_n + r * ld + pb;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      float va[4], vb[4];
#pragma unroll
      for (int sl = 0; sl < 4; ++sl) {
        const int cp = acomp[ks][sl];
        float xa = 0.f, xb = 0.f;
        if (cp >= 0) {
          const float2 fa = pa < W ? base_a[aoff[ks][sl]] : make_float2(0.f, 0.f);
          const float2 fb = pb < W ? base_b[aoff[ks][sl]] : make_float2(0.f, 0.f);
          xa = (cp & 1) ? fa.y : fa.x;
          xb = (cp & 1) ? fb.y : fb.x;
          if (MODE == 1) {  // BF16 term part = cp >> 1 of the FP32 value
            const int part = cp >> 1;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              if (part > q) {
                xa -= bf(__float2bfloat16_rn(xa));
                xb -= bf(__float2bfloat16_rn(xb));
              }
            }
          }
        }
        va[sl] = xa;
        vb[sl] = xb;
      }
      uint32_t afr[4];
      afr[0] = pack_bf2(va[0], va[1]);  // row gid, k 2tig, 2tig+1
      afr[1] = pack_bf2(vb[0], vb[1]);  // row gid+8
      afr[2] = pack_bf2(va[2], va[3]);  // row gid, k 2tig+8, +9
      afr[3] = pack_bf2(vb[2], vb[3]);  // row gid+8
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const uint2 bb = s_f[(ks * 8 + nt) * 32 + lane];
        mma_bf16_16816(acc[nt], afr, bb.x, bb.y);
      }
    }
    // stage the 16 x 64 result (mode 0: ReLU) as BF16
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float v0 = acc[nt][0], v1 = acc[nt][1], v2 = acc[nt][2], v3 = acc[nt][3];
      if (MODE == 0) {
        v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); v2 = fmaxf(v2, 0.f); v3 = fmaxf(v3, 0.f);
      }
      *reinterpret_cast<uint32_t*>(so + gid * k2Ld + 8 * nt + 2 * tig) = pack_bf2(v0, v1);
      *reinterpret_cast<uint32_t*>(so + (gid + 8) * k2Ld + 8 * nt + 2 * tig) = pack_bf2(v2, v3);
    }
    __syncwarp();
    // 16 pixels x 8 chunks of 16 bytes: four chunks per lane, whole 128-byte pixel rows per 8 lanes
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = q * 32 + lane, m = idx >> 3, ch = idx & 7;
      const int px = w0 + m;
      if (px < W) {
        uint4 v = *reinterpret_cast<const uint4*>(so + m * k2Ld + ch * 8);
        if (MODE == 1) {
          const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mk[q]);
          __nv_bfloat16* vb = reinterpret_cast<__nv_bfloat16*>(&v);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (!(bf(mb[e]) > 0.f)) vb[e] = __float2bfloat16_rn(0.f);
        }
        reinterpret_cast<uint4*>(out + (prow + px) * CH)[ch] = v;
      }
    }
    __syncwarp();
  }
}

// --------------------------------------------------- weight gradients (CUDA cores)
// Small layers (partials per CTA, reduced later):
//  L1 (first):  gw[co][c][tap] = sum_p g1[p][co] * xr[p + s][c],  gb[co] = sum_p g1[p][co]
//  L5 (last):   gw[co][ci][tap] = sum_p g5[p][co] * a4[p + s][ci], gb[co] = sum_p g5[p][co]
// Thread j < 64 of each of the four groups owns the 64-channel index (co for
// L1, ci for L5) and 18 (+1) sums over a quarter of each row's pixels, all
// operands in shared memory; the groups are added in fixed order.
constexpr int kSmallOut = CH * 18 + CH;  // 1152 weights + up to 64 biases

__device__ void small_partial_out(float (&acc)[2][9], float bacc, int last, float* out) {
  __shared__ float s_red[4][CH * 19];
  const int j = threadIdx.x & 63, grp = threadIdx.x >> 6;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int t = 0; t < 9; ++t) s_red[grp][j * 19 + c * 9 + t] = acc[c][t];
  s_red[grp][j * 19 + 18] = bacc;
  __syncthreads();
  for (int i = threadIdx.x; i < CH * 19; i += blockDim.x) {
    const float v = ((s_red[0][i] + s_red[1][i]) + s_red[2][i]) + s_red[3][i];
    const int jj = i / 19, r = i % 19;
    if (r == 18) {
      out[CH * 18 + jj] = v;
    } else {
      const int c = r / 9, tap = r % 9;
      out[!last ? ((jj * 2 + c) * 9 + tap) : ((c * CH + jj) * 9 + tap)] = v;
    }
  }
}

// A CTA takes kSmallRows consecutive rows of one slice; the sums of all its rows accumulate in
// registers (one partial per CTA).  Thread j < 64 of group g (of four) owns channel j and the
// pixel range [g W4, (g + 1) W4) of every row, walked with a 3 x 3 window kept in registers (one
// new window column per pixel).  The 3-row halo source sits in a ring of three row slots
// (row yy in slot (yy + 3) mod 3, one new row staged per output row), zero outside the image.
constexpr int kSmallRows = 4;

__device__ __forceinline__ int ring_slot(int yy) { return (yy + 3) % 3; }

// L1: U = g1 row h [W][64] (bf16), V = bf16-rounded x, ring of rows [3][W+2] (float2).
__global__ void __launch_bounds__(256) k_wgrad_l1(int B, int H, int W, const __nv_bfloat16* g1,
                                                  const float2* x, float* partial) {
  extern __shared__ __align__(16) uint8_t dsm[];
  __nv_bfloat16* su = reinterpret_cast<__nv_bfloat16*>(dsm);
  float2* sv = reinterpret_cast<float2*>(dsm + (((size_t)W * CH * 2 + 15) & ~(size_t)15));
  const int nrb = (H + kSmallRows - 1) / kSmallRows;
  const int b = blockIdx.x / nrb, h0 = (blockIdx.x % nrb) * kSmallRows, h1 = min(h0 + kSmallRows, H);
  auto stage_x = [&](int yy) {  // x row yy (zero outside) into its ring slot, columns -1 .. W
    float2* d = sv + ring_slot(yy) * (W + 2);
    for (int i = threadIdx.x; i < W + 2; i += blockDim.x) {
      const int xx = i - 1;
      float2 v = make_float2(0.f, 0.f);
      if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
        v = x[((size_t)b * H + yy) * W + xx];
        v = make_float2(bf(__float2bfloat16_rn(v.x)), bf(__float2bfloat16_rn(v.y)));
      }
      d[i] = v;
    }
  };
  stage_x(h0 - 1);
  stage_x(h0);
  const int j = threadIdx.x & 63, grp = threadIdx.x >> 6;
  const int W4 = (W + 3) / 4, wa = min(W, grp * W4), wb = min(W, wa + W4);
  float2 acc2[9];  // (input channel 0, 1) of each tap
  float bacc = 0.f;
#pragma unroll
  for (int t = 0; t < 9; ++t) acc2[t] = make_float2(0.f, 0.f);
  for (int h = h0; h < h1; ++h) {
    __syncthreads();  // the slots and the g1 row of the previous row are no longer read
    const __nv_bfloat16* src = g1 + ((size_t)b * H + h) * W * CH;
    for (int i = threadIdx.x; i < W * 8; i += blockDim.x) cp_async16(su + i * 8, src + i * 8, true);
    cp_async_commit();
    stage_x(h + 1);
    cp_async_wait0();
    __syncthreads();
    const float2* r0 = sv + ring_slot(h - 1) * (W + 2);
    const float2* r1 = sv + ring_slot(h) * (W + 2);
    const float2* r2 = sv + ring_slot(h + 1) * (W + 2);
    if (wa < wb) {
      // window columns w - 1, w, w + 1 (image) = slot columns w, w + 1, w + 2; the two input
      // channels of a tap as one packed FP32x2 FMA
      float2 c0[3] = {r0[wa], r1[wa], r2[wa]};
      float2 c1[3] = {r0[wa + 1], r1[wa + 1], r2[wa + 1]};
#pragma unroll 3
      for (int w = wa; w < wb; ++w) {
        const float2 c2[3] = {r0[w + 2], r1[w + 2], r2[w + 2]};
        const float u = bf(su[w * CH + j]);
        const float2 uu = make_float2(u, u);
        bacc += u;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          acc2[dy * 3 + 0] = __ffma2_rn(uu, c0[dy], acc2[dy * 3 + 0]);
          acc2[dy * 3 + 1] = __ffma2_rn(uu, c1[dy], acc2[dy * 3 + 1]);
          acc2[dy * 3 + 2] = __ffma2_rn(uu, c2[dy], acc2[dy * 3 + 2]);
        }
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          c0[dy] = c1[dy];
          c1[dy] = c2[dy];
        }
      }
    }
  }
  __syncthreads();
  float acc[2][9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    acc[0][t] = acc2[t].x;
    acc[1][t] = acc2[t].y;
  }
  small_partial_out(acc, bacc, 0, partial + (size_t)blockIdx.x * kSmallOut);
}

// L5: U = a4, ring of rows [3][W+2][64] (bf16), V = g5 row h [W] (float2).
__global__ void __launch_bounds__(256) k_wgrad_l5(int B, int H, int W, const __nv_bfloat16* a4,
                                                  const float2* g5, float* partial) {
  extern __shared__ __align__(16) uint8_t dsm[];
  __nv_bfloat16* su = reinterpret_cast<__nv_bfloat16*>(dsm);
  float2* sv = reinterpret_cast<float2*>(dsm + (size_t)3 * (W + 2) * CH * 2);
  const int nrb = (H + kSmallRows - 1) / kSmallRows;
  const int b = blockIdx.x / nrb, h0 = (blockIdx.x % nrb) * kSmallRows, h1 = min(h0 + kSmallRows, H);
  auto stage_a = [&](int yy) {  // a4 row yy (zero outside) into its ring slot, columns -1 .. W
    __nv_bfloat16* d = su + (size_t)ring_slot(yy) * (W + 2) * CH;
    for (int i = threadIdx.x; i < (W + 2) * 8; i += blockDim.x) {
      const int q = i & 7, px = i >> 3, xx = px - 1;
      const bool ok = yy >= 0 && yy < H && xx >= 0 && xx < W;
      cp_async16(d + (px * 8 + q) * 8, a4 + (ok ? (((size_t)b * H + yy) * W + xx) * CH + q * 8 : 0), ok);
    }
  };
  stage_a(h0 - 1);
  stage_a(h0);
  const int j = threadIdx.x & 63, grp = threadIdx.x >> 6;
  const int W4 = (W + 3) / 4, wa = min(W, grp * W4), wb = min(W, wa + W4);
  float2 acc2[9];  // (output channel 0, 1) of each tap
  float bacc = 0.f;
#pragma unroll
  for (int t = 0; t < 9; ++t) acc2[t] = make_float2(0.f, 0.f);
  for (int h = h0; h < h1; ++h) {
    __syncthreads();  // the slot of row h - 2 and the g5 row of the previous row are no longer read
    stage_a(h + 1);
    cp_async_commit();
    for (int i = threadIdx.x; i < W; i += blockDim.x) sv[i] = g5[((size_t)b * H + h) * W + i];
    cp_async_wait0();
    __syncthreads();
    const __nv_bfloat16* r0 = su + (size_t)ring_slot(h - 1) * (W + 2) * CH + j;
    const __nv_bfloat16* r1 = su + (size_t)ring_slot(h) * (W + 2) * CH + j;
    const __nv_bfloat16* r2 = su + (size_t)ring_slot(h + 1) * (W + 2) * CH + j;
    if (wa < wb) {
      float c0[3] = {bf(r0[wa * CH]), bf(r1[wa * CH]), bf(r2[wa * CH])};
      float c1[3] = {bf(r0[(wa + 1) * CH]), bf(r1[(wa + 1) * CH]), bf(r2[(wa + 1) * CH])};
#pragma unroll 3
      for (int w = wa; w < wb; ++w) {
        const float c2[3] = {bf(r0[(w + 2) * CH]), bf(r1[(w + 2) * CH]), bf(r2[(w + 2) * CH])};
        const float2 v = sv[w];
        if (j < 2) bacc += (j == 0) ? v.x : v.y;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          acc2[dy * 3 + 0] = __ffma2_rn(v, make_float2(c0[dy], c0[dy]), acc2[dy * 3 + 0]);
          acc2[dy * 3 + 1] = __ffma2_rn(v, make_float2(c1[dy], c1[dy]), acc2[dy * 3 + 1]);
          acc2[dy * 3 + 2] = __ffma2_rn(v, make_float2(c2[dy], c2[dy]), acc2[dy * 3 + 2]);
        }
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          c0[dy] = c1[dy];
          c1[dy] = c2[dy];
        }
      }
    }
  }
  __syncthreads();
  float acc[2][9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    acc[0][t] = acc2[t].x;
    acc[1][t] = acc2[t].y;
  }
  small_partial_out(acc, bacc, 1, partial + (size_t)blockIdx.x * kSmallOut);
}

// Deterministic sums over chunks, added to the caller's gradient buffers.  A
// CTA owns 32 consecutive columns; its eight warps each sum every eighth chunk
// in increasing order, and the eight results are added in warp order.
__device__ __forceinline__ float colsum8(const float* base, size_t stride, int nchunks, bool valid) {
  __shared__ float s_part[8][32];
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
  float s = 0.f;
  if (valid) {
    int c = wg;
    for (; c + 7 * 8 < nchunks; c += 8 * 8) {  // eight loads in flight, added in chunk order
      float v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = __ldcg(base + (size_t)(c + 8 * k) * stride);
#pragma unroll
      for (int k = 0; k < 8; ++k) s += v[k];
    }
    for (; c < nchunks; c += 8) s += __ldcg(base + (size_t)c * stride);
  }
  s_part[wg][lane] = s;
  __syncthreads();
  float t = 0.f;
  if (wg == 0)
    for (int k = 0; k < 8; ++k) t += s_part[k][lane];
  return t;
}

// Small layers: column i < nw is weight i, nw <= i < nw + nb is bias i - nw (at boff).
__global__ void __launch_bounds__(256) k_reduce_partials(const float* partial, int nchunks, int stride, int nw,
                                                         float* gw, int nb, int boff, float* gb) {
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const bool valid = i < nw + nb;
  const int src = valid ? ((i < nw) ? i : boff + (i - nw)) : 0;
  const float s = colsum8(partial + src, stride, nchunks, valid);
  if (threadIdx.x < 32 && valid) {
    if (i < nw) gw[i] += s;
    else gb[i - nw] += s;
  }
}

// 64 -> 64 layer weight gradient on tcgen05 (BF16 operands, FP32 accumulation in TMEM):
//   gw[co][ci][tap] = sum_p g[p][co] * a[p + s_tap][ci],  gb[co] = sum_p g[p][co],
// a contraction over pixels.  Work items are row segments (slice b, row h, pixels
// w0 .. w0 + 127); each CTA takes a contiguous range of them and keeps its sums in TMEM until the
// end.  Per item a TMA box brings activation rows h-1, h, h+1 (pixels w0-1 .. w0+134, zero
// outside the image) and one box the gradient row h; both are channels-last with 128-byte rows,
// i.e. MN-major operands with K = pixels.  For each 16-pixel step and horizontal tap dx:
//   MMA a: A = [row h-1 | row h] (two 64-channel blocks one row apart, M = 128), B = g row h
//          -> TMEM lanes 0-63 accumulate tap (0, dx), lanes 64-127 tap (1, dx);
//   MMA b: A = [row h+1 | ones] -> lanes 0-63 tap (2, dx), lanes 64-127 the bias sums.
// The pixel offset dx is a start-address offset of 128 bytes (the swizzle follows the address
// bits).  Warp 4 (one lane) issues TMA and MMAs through a three-slot pipeline; warps 0-3 read the
// accumulators once at the end and write the CTA's partial sums [tap][co][ci] and bias [co],
// which k_reduce_wgrad64 adds over CTAs in fixed order.
constexpr int WG_SEG = 128;
constexpr int WG_ROWPX = 136;                 // staged pixels per activation row (130 used)
constexpr int WG_ROWB = WG_ROWPX * 128;       // 17408
constexpr int WG_ACT = 3 * WG_ROWB;
constexpr int WG_GB = WG_SEG * 128;
constexpr int WG_STAGE = WG_ACT + WG_GB;      // 68608 (1 KB multiple)
constexpr int WG_NST = 3;
constexpr int WG_ONES = WG_NST * WG_STAGE;
constexpr int WG_ONES_BYTES = 130 * 128;      // covers the offsets (16 kk + dx) + 15 rows
constexpr int WG_BAR = WG_ONES + WG_ONES_BYTES;
constexpr int WG_NBARS = 2 * WG_NST + 1;
constexpr int WG_SMEM = WG_BAR + WG_NBARS * 8 + 16 + 1024;
constexpr int WG_THREADS = 160;
constexpr int kWgMaxParts = 256;              // partial-sum slots (one per CTA, CTAs <= SM count)

struct WgArgs {
  int B, H, W, nseg, items;
  float* partial;
  int* status;
};

__device__ __forceinline__ void wg_item(int it, int H, int nseg, int& b, int& h, int& seg) {
  h = it % H;
  const int t = it / H;
  seg = t % nseg;
  b = t / nseg;
}

__global__ void __launch_bounds__(WG_THREADS, 1)
k_wgrad64(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap gmap, const WgArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + WG_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + WG_NST;
  uint64_t* done = bars + 2 * WG_NST;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + WG_NBARS);
  int* s_err = reinterpret_cast<int*>(s_tmem + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = (int)(((long long)blockIdx.x * a.items) / gridDim.x);
  const int i1 = (int)(((long long)(blockIdx.x + 1) * a.items) / gridDim.x);
  const int n = i1 - i0;

  if (tid == 0) {
    for (int k = 0; k < WG_NST; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    mbar_init(done, 1);
    *s_err = 0;
    fence_mbar_init();
  }
  {  // the ones block (BF16 1.0), read by the tensor cores through the async proxy
    uint4* o = reinterpret_cast<uint4*>(smem + WG_ONES);
    for (int i = tid; i < WG_ONES_BYTES / 16; i += blockDim.x) o[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    fence_proxy_async();
  }
  if (warp == 0) {
    tmem_alloc(s_tmem, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  griddep_wait();  // the activations and gradient rows, and the partial sums written below
  griddep_release();

  int tma_issued = 0, mma_issued = 0;
  if (warp == 4) {
    if (lane == 0 && n > 0) {
      const uint32_t idesc = umma_idesc_bf16_mn(128, CH);
      const uint32_t ones = smem_u32(smem + WG_ONES);
      auto load = [&](int it, int s) {
        int b, h, seg;
        wg_item(it, a.H, a.nseg, b, h, seg);
        uint8_t* st = smem + s * WG_STAGE;
        mbar_expect_tx(&full[s], WG_STAGE);
        tma_load_4d(st, &amap, 0, seg * WG_SEG - 1, h - 1, b, &full[s]);
        tma_load_4d(st + WG_ACT, &gmap, 0, seg * WG_SEG, h, b, &full[s]);
      };
      bool ok = true;
      const int pre = n < 2 ? n : 2;
      for (int j = 0; j < pre; ++j) {
        load(i0 + j, j);
        ++tma_issued;
      }
      for (int i = 0; i < n && ok; ++i) {
        const int s = i % WG_NST;
        ok = mbar_wait(&full[s], (i / WG_NST) & 1);
        if (!ok) break;
        tc_fence_after();
        int b, h, seg;
        wg_item(i0 + i, a.H, a.nseg, b, h, seg);
        const int rem = a.W - seg * WG_SEG;
        const int nk = rem >= WG_SEG ? WG_SEG / 16 : (rem + 15) / 16;
        const uint32_t act = smem_u32(smem + s * WG_STAGE);
        const uint32_t gro = act + WG_ACT;
        const uint32_t lbo_b = ones - (act + 2 * WG_ROWB);
        for (int kk = 0; kk < nk; ++kk) {
          const uint64_t bd = umma_desc_mn_sw128(gro + kk * 2048, 1024);
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const uint32_t off = (uint32_t)(kk * 16 + dx) * 128;
            const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
            umma_bf16(tmem + dx * 128, umma_desc_mn_sw128(act + off, WG_ROWB), bd, idesc, acc);
            umma_bf16(tmem + dx * 128 + 64, umma_desc_mn_sw128(act + 2 * WG_ROWB + off, lbo_b), bd, idesc, acc);
          }
        }
        umma_commit(&empty[s]);
        ++mma_issued;
        if (i + 2 < n) {  // refill the slot of item i - 1 with item i + 2
          const int s2 = (i + 2) % WG_NST;
          if (i >= 1) ok = mbar_wait(&empty[s2], ((i - 1) / WG_NST) & 1);
          if (!ok) break;
          load(i0 + i + 2, s2);
          ++tma_issued;
        }
      }
      if (ok) {
        umma_commit(done);
      } else {
        atomicExch(s_err, 1);
        mbar_arrive(done);
      }
    }
  } else if (n > 0) {
    // epilogue: TMEM lane m = 32 warp + lane
    const bool ok = mbar_wait(done, 0);
    tc_fence_after();
    if (!ok) atomicExch(s_err, 1);
    const bool write = ok && *reinterpret_cast<volatile int*>(s_err) == 0;
    const int m = warp * 32 + lane;
    float* out = a.partial + (size_t)blockIdx.x * 9 * CH * CH;
#pragma unroll 1
    for (int q = 0; q < 6; ++q) {
      const int dx = q >> 1, half = q & 1;
      float v[64];
      tmem_ld64(tmem + ((uint32_t)(warp * 32) << 16) + dx * 128 + half * 64, v);
      if (!write) continue;
      if (half == 1 && m >= 64) {  // bias sums (identical in every lane of this block)
        if (dx == 0 && m == 64) {
          float* ob = a.partial + (size_t)gridDim.x * 9 * CH * CH + (size_t)blockIdx.x * CH;
#pragma unroll
          for (int co = 0; co < CH; ++co) ob[co] = v[co];
        }
        continue;
      }
      const int dy = half == 0 ? (m >> 6) : 2;
      const int ci = m & 63;
      float* o = out + (size_t)(dy * 3 + dx) * CH * CH + ci;
#pragma unroll
      for (int co = 0; co < CH; ++co) o[co * CH] = v[co];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*s_err && tid == 4 * 32) {
    set_status(a.status, SENSE_STATUS_DEVICE_TIMEOUT);
    // bounded drain of the copies and MMAs still in flight before the memory is released
    for (int j = tma_issued > WG_NST ? tma_issued - WG_NST : 0; j < tma_issued; ++j)
      mbar_wait(&full[j % WG_NST], (j / WG_NST) & 1, 1u << 20);
    if (mma_issued > 0) {
      const int j = mma_issued - 1;
      mbar_wait(&empty[j % WG_NST], (j / WG_NST) & 1, 1u << 20);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// Sum the 64x64-layer partials over chunks in fixed order into gw [co][ci][tap] and gb.
// 64x64 layers: columns (tap, co, ci) of the per-chunk [9][64][64] partials, then the biases.
__global__ void __launch_bounds__(256) k_reduce_wgrad64(const float* partial, int nchunks, float* gw,
                                                        float* gb) {
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int nw = CH * CH * 9;
  const bool valid = i < nw + CH;
  float s;
  if (i < nw || !valid) {
    s = colsum8(partial + (valid ? i : 0), (size_t)nw, nchunks, valid);
  } else {
    s = colsum8(partial + (size_t)nchunks * nw + (i - nw), CH, nchunks, true);
  }
  if (threadIdx.x < 32 && valid) {
    if (i < nw) {
      const int tap = i / (CH * CH), co = (i / CH) % CH, ci = i % CH;
      gw[(co * CH + ci) * 9 + tap] += s;
    } else {
      gb[i - nw] += s;
    }
  }
}

// ------------------------------------------------------------ host helpers
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Tensor map over a BF16 [B][H][W][64] activation; box 8 ch x 130 px x 3 rows x 1 slice.
// 4-D map {channel, pixel, row, slice} of a channels-last BF16 tensor, 128-byte swizzle; boxes of
// box_px pixels x box_rows rows (the convolution halo by default).
int make_act_map(CUtensorMap* m, const void* base, int B, int H, int W, int box_px = TILE_M, int box_rows = 3) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return SENSE_ECUDA;
  const cuuint64_t dims[4] = {(cuuint64_t)CH, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)CH * 2, (cuuint64_t)W * CH * 2, (cuuint64_t)H * W * CH * 2};
  const cuuint32_t box[4] = {CH, (cuuint32_t)box_px, (cuuint32_t)box_rows, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box,
                         es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SENSE_OK : SENSE_ECUDA;
}

int g_num_sms = 0;
constexpr int kMaxW = 512;  // widest image the denoiser kernels take (shared-memory tiles)
int wl1_smem(int W) { return (int)((((size_t)W * CH * 2 + 15) & ~(size_t)15) + 3 * (W + 2) * 8); }
int wl5_smem(int W) { return 3 * (W + 2) * CH * 2 + W * 8; }

int conv_prepare() {
  static int state = 0;  // 0 unknown, 1 ok, -1 failed
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (state == 0) {
    int dev = 0;
    state = (cudaGetDevice(&dev) == cudaSuccess &&
             cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
             cudaFuncSetAttribute(k_conv64<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ConvLayout<64>::SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_conv64<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ConvLayout<16>::SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_wgrad64, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(k_2to64<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem(kMaxW)) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(k_2to64<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem(kMaxW)) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(k_wgrad_l1, cudaFuncAttributeMaxDynamicSharedMemorySize, wl1_smem(kMaxW)) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(k_wgrad_l5, cudaFuncAttributeMaxDynamicSharedMemorySize, wl5_smem(kMaxW)) ==
                 cudaSuccess)
                ? 1
                : -1;
  }
  return state == 1 ? SENSE_OK : SENSE_ECUDA;
}

int launch_conv64(const __nv_bfloat16* in, const __nv_bfloat16* wpack, const float* bias,
                  const __nv_bfloat16* aprev, __nv_bfloat16* out, int mode, int B, int H, int W,
                  int* status, cudaStream_t st, const float2* res = nullptr, float2* out2 = nullptr) {
  const bool two = mode >= 2;  // 64 -> 2 layers (NOUT = 16)
  const int halo_px = two ? ConvLayout<16>::HALO_PX : ConvLayout<64>::HALO_PX;
  const int tile_out = two ? ConvLayout<16>::TILE_OUT : ConvLayout<64>::TILE_OUT;
  CUtensorMap map;
  if (int e = make_act_map(&map, in, B, H, W, halo_px, 3)) return e;
  ConvArgs a;
  a.B = B; a.H = H; a.W = W; a.ntw = (W + tile_out - 1) / tile_out;
  a.wpack = wpack; a.bias = bias; a.aprev = aprev; a.out = out; a.mode = mode; a.status = status;
  a.res = res; a.out2 = out2;
  const int ntiles = B * H * a.ntw;
  const int grid = ntiles < g_num_sms ? ntiles : g_num_sms;
  // programmatic stream serialisation: the prologue overlaps the previous kernel's tail
  cudaError_t e;
  if (mode >= 2) {  // 64 -> 2 layers
    prof_mark("dn_64to2", st, false);
    e = launch_pdl(k_conv64<16>, dim3(grid), dim3(CONV_THREADS), ConvLayout<16>::SMEM, st, map, a);
    prof_mark("dn_64to2", st, true);
  } else {
    prof_mark("conv64_tc", st, false);
    e = launch_pdl(k_conv64<64>, dim3(grid), dim3(CONV_THREADS), ConvLayout<64>::SMEM, st, map, a);
    prof_mark("conv64_tc", st, true);
  }
  prof_count(1);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

size_t up256(size_t n) { return (n + 255) & ~(size_t)255; }

// Weight gradient of a 64 -> 64 layer into per-CTA partial sums (at most max_parts CTAs).
int launch_wgrad64(const __nv_bfloat16* g, const __nv_bfloat16* act, float* partial, int max_parts, int B, int H,
                   int W, int* status, cudaStream_t st, int* nparts) {
  CUtensorMap amap, gmap;
  if (int e = make_act_map(&amap, act, B, H, W, WG_ROWPX, 3)) return e;
  if (int e = make_act_map(&gmap, g, B, H, W, WG_SEG, 1)) return e;
  WgArgs a;
  a.B = B; a.H = H; a.W = W; a.nseg = (W + WG_SEG - 1) / WG_SEG;
  a.items = B * H * a.nseg;
  a.partial = partial; a.status = status;
  int grid = a.items < g_num_sms ? a.items : g_num_sms;
  if (grid > max_parts) grid = max_parts;
  *nparts = grid;
  prof_mark("wgrad64", st, false);
  const cudaError_t e = launch_pdl(k_wgrad64, dim3(grid), dim3(WG_THREADS), WG_SMEM, st, amap, gmap, a);
  prof_mark("wgrad64", st, true);
  prof_count(1);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

struct DnLayout {
  size_t wf[3], wd[3], ts[2], tf[2], act[4], g[2], zout, part_small, part64, status, total;
  int nch_small, nch64;
};

DnLayout dn_layout(int B, int H, int W) {
  DnLayout L;
  const size_t act = up256((size_t)B * H * W * CH * 2);
  L.nch_small = B * ((H + kSmallRows - 1) / kSmallRows);
  L.nch64 = std::min(B * H * ((W + WG_SEG - 1) / WG_SEG), kWgMaxParts);
  size_t o = 0;
  for (int i = 0; i < 3; ++i) { L.wf[i] = o; o += up256(WPACK_BYTES); }
  for (int i = 0; i < 3; ++i) { L.wd[i] = o; o += up256(WPACK_BYTES); }
  for (int i = 0; i < 2; ++i) { L.ts[i] = o; o += up256(WP16_BYTES); }
  for (int i = 0; i < 2; ++i) { L.tf[i] = o; o += up256((size_t)(i == 0 ? 2 : 4) * 8 * 32 * 2 * 4); }
  for (int i = 0; i < 4; ++i) { L.act[i] = o; o += act; }
  for (int i = 0; i < 2; ++i) { L.g[i] = o; o += act; }
  L.zout = o; o += up256((size_t)B * H * W * 8);  // the block output z of an unrolled step
  L.part_small = o; o += up256((size_t)L.nch_small * kSmallOut * 4);
  // two sets: the reduction of one layer's partials (side stream) overlaps the next layer's sums
  L.part64 = o; o += 2 * up256(((size_t)L.nch64 * 9 * CH * CH + (size_t)L.nch64 * CH) * 4);
  L.status = o; o += 256;
  L.total = o;
  return L;
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }


int check_common(int kind, const void* weights, const void* x, void* ws, size_t ws_bytes, int B, int H,
                 int W) {
  if (kind != SENSE_DENOISER_MODL) return SENSE_EUNSUPPORTED;
  if (B <= 0 || H <= 0 || W <= 0) return SENSE_EINVAL_SHAPE;
  if (W > kMaxW || (W & 1)) return SENSE_EUNSUPPORTED;
  if (!weights || !x || !ws || !al16(weights) || !al16(x) || ((uintptr_t)ws & 255u)) return SENSE_EINVAL_PTR;
  if (ws_bytes < dn_layout(B, H, W).total) return SENSE_EWORKSPACE;
  return conv_prepare();
}

int forward_impl(const float* wts, const float2* x, float2* out, uint8_t* ws, int B, int H, int W,
                 cudaStream_t st) {
  const DnLayout L = dn_layout(B, H, W);
  const ModlOffsets o = modl_offsets();
  __nv_bfloat16* act[4];
  for (int i = 0; i < 4; ++i) act[i] = reinterpret_cast<__nv_bfloat16*>(ws + L.act[i]);
  int* status = reinterpret_cast<int*>(ws + L.status);
  {
    PackArgs pa;
    for (int l = 0; l < 3; ++l) {
      pa.w[l] = wts + o.w[l + 1];
      pa.fwd[l] = reinterpret_cast<__nv_bfloat16*>(ws + L.wf[l]);
      pa.dgr[l] = reinterpret_cast<__nv_bfloat16*>(ws + L.wd[l]);
    }
    prof_mark("dn_pack", st, false);
    pa.w1 = wts + o.w[0];
    pa.w5 = wts + o.w[4];
    pa.t5 = reinterpret_cast<__nv_bfloat16*>(ws + L.ts[0]);
    pa.t1 = reinterpret_cast<__nv_bfloat16*>(ws + L.ts[1]);
    pa.f1 = reinterpret_cast<uint32_t*>(ws + L.tf[0]);
    pa.f5 = reinterpret_cast<uint32_t*>(ws + L.tf[1]);
    launch_pdl(k_pack64, dim3((9 * 8 * CH * 8 + 255) / 256, 10), dim3(256), 0, st, pa);
    prof_mark("dn_pack", st, true);
  }
  const size_t npx = (size_t)B * H * W;
  prof_mark("dn_2to64", st, false);
  launch_pdl(k_2to64<0>, dim3((unsigned)(B * ((H + k2Rows - 1) / k2Rows))), dim3(k2Threads), k2_smem(W), st,
      B, H, W, x, reinterpret_cast<const uint32_t*>(ws + L.tf[0]), wts + o.b[0], nullptr, act[0]);
  prof_mark("dn_2to64", st, true);
  for (int l = 0; l < 3; ++l)
    if (int e = launch_conv64(act[l], reinterpret_cast<__nv_bfloat16*>(ws + L.wf[l]), wts + o.b[l + 1],
                              nullptr, act[l + 1], 0, B, H, W, status, st))
      return e;
  if (out)  // last layer on the tensor cores: out = x + b5 + conv(a4) (two of 16 MMA columns used)
    if (int e = launch_conv64(act[3], reinterpret_cast<const __nv_bfloat16*>(ws + L.ts[0]), wts + o.b[4],
                              nullptr, nullptr, 2, B, H, W, status, st, x, out))
      return e;
  prof_count(2);  // packing, first layer (convolutions counted apart)
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

}  // namespace

// z = D(x_t) of an unrolled MoDL step, kept in its denoiser workspace beside the activations.
float2* modl_zout(void* ws, int B, int H, int W) {
  return reinterpret_cast<float2*>(static_cast<uint8_t*>(ws) + dn_layout(B, H, W).zout);
}

extern "C" {

size_t denoiser_workspace_bytes(int kind, int B, int H, int W) {
  if (kind == SENSE_DENOISER_VARNET) return vn_denoiser_bytes(B, H, W);
  if (kind != SENSE_DENOISER_MODL || B <= 0 || H <= 0 || W <= 0) return 0;
  return dn_layout(B, H, W).total;
}

int denoiser_param_count(int kind) {
  if (kind == SENSE_DENOISER_VARNET) return varnet_param_count();
  return kind == SENSE_DENOISER_MODL ? modl_offsets().total : 0;
}

int denoiser_workspace_offsets(int kind, int B, int H, int W, size_t* act_offsets /*[4]*/,
                               size_t* grad_offsets /*[2]*/) {
  if (kind != SENSE_DENOISER_MODL || B <= 0 || H <= 0 || W <= 0) return SENSE_EINVAL_ARG;
  const DnLayout L = dn_layout(B, H, W);
  if (act_offsets)
    for (int i = 0; i < 4; ++i) act_offsets[i] = L.act[i];
  if (grad_offsets)
    for (int i = 0; i < 2; ++i) grad_offsets[i] = L.g[i];
  return SENSE_OK;
}

int denoiser_forward(int kind, const float* weights, const void* x, void* out, void* ws, size_t ws_bytes,
                     int B, int H, int W, void* stream) {
  if (kind == SENSE_DENOISER_VARNET)
    return vn_denoiser_forward(weights, x, out, ws, ws_bytes, B, H, W, static_cast<cudaStream_t>(stream));
  if (int e = check_common(kind, weights, x, ws, ws_bytes, B, H, W)) return e;
  if (!out || !al16(out) || out == x) return SENSE_EINVAL_PTR;
  return forward_impl(weights, static_cast<const float2*>(x), static_cast<float2*>(out),
                      static_cast<uint8_t*>(ws), B, H, W, static_cast<cudaStream_t>(stream));
}

int denoiser_backward(int kind, const float* weights, const void* x, const void* grad_out, void* grad_x,
                      float* grad_weights, void* ws, size_t ws_bytes, int B, int H, int W, int recompute,
                      void* stream) {
  if (kind == SENSE_DENOISER_VARNET)  // always recomputes K x (the workspace keeps no forward state)
    return vn_denoiser_backward(weights, x, grad_out, grad_x, grad_weights, ws, ws_bytes, B, H, W,
                                static_cast<cudaStream_t>(stream));
  if (int e = check_common(kind, weights, x, ws, ws_bytes, B, H, W)) return e;
  if (!grad_out || !grad_x || !grad_weights || !al16(grad_out) || !al16(grad_x) || !al16(grad_weights) ||
      grad_x == grad_out)
    return SENSE_EINVAL_PTR;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* w8 = static_cast<uint8_t*>(ws);
  const DnLayout L = dn_layout(B, H, W);
  const ModlOffsets o = modl_offsets();
  const float2* xx = static_cast<const float2*>(x);
  const float2* go = static_cast<const float2*>(grad_out);
  if (recompute)
    if (int e = forward_impl(weights, xx, nullptr, w8, B, H, W, st)) return e;
  __nv_bfloat16* act[4];
  for (int i = 0; i < 4; ++i) act[i] = reinterpret_cast<__nv_bfloat16*>(w8 + L.act[i]);
  __nv_bfloat16* gbuf[2] = {reinterpret_cast<__nv_bfloat16*>(w8 + L.g[0]),
                            reinterpret_cast<__nv_bfloat16*>(w8 + L.g[1])};
  float* ps = reinterpret_cast<float*>(w8 + L.part_small);
  float* p64 = reinterpret_cast<float*>(w8 + L.part64);
  int* status = reinterpret_cast<int*>(w8 + L.status);
  // (the input-gradient weight tables were packed by the forward pass that precedes every backward)
  // The weight-gradient sums of the 2-channel layers and every fixed-order reduction run on a
  // side stream beside the data-gradient chain (CUDA cores and memory against tensor cores)
  SideSet* ss = nullptr;
  if (int e = side_set(&ss)) return e;
  cudaStream_t sd = ss->s[0];
  const size_t p64_set = up256(((size_t)L.nch64 * 9 * CH * CH + (size_t)L.nch64 * CH) * 4) / sizeof(float);
  // fork: the side stream sees the activations, the output gradient and the zeroed sums
  if (int e = stream_after(*ss, st, sd)) return e;
  // last layer: input gradient (masked by a4 > 0) on the caller's stream, weight gradient beside it
  prof_mark("dn_2to64", st, false);
  launch_pdl(k_2to64<1>, dim3((unsigned)(B * ((H + k2Rows - 1) / k2Rows))), dim3(k2Threads), k2_smem(W), st,
      B, H, W, go, reinterpret_cast<const uint32_t*>(w8 + L.tf[1]), nullptr, act[3], gbuf[0]);
  prof_mark("dn_2to64", st, true);
  prof_mark("dn_wgrad_small", sd, false);
  k_wgrad_l5<<<L.nch_small, 256, wl5_smem(W), sd>>>(B, H, W, act[3], go, ps);
  prof_mark("dn_wgrad_small", sd, true);
  prof_mark("dn_reduce", sd, false);
  k_reduce_partials<<<(2 * CH * 9 + 2 + 31) / 32, 256, 0, sd>>>(ps, L.nch_small, kSmallOut, 2 * CH * 9,
                                                                 grad_weights + o.w[4], 2, CH * 18,
                                                                 grad_weights + o.b[4]);
  prof_mark("dn_reduce", sd, true);
  // 64 -> 64 layers 4, 3, 2 (index l = 2, 1, 0 of the packed set); partial set l & 1
  int cur = 0;
  for (int l = 2; l >= 0; --l) {
    const __nv_bfloat16* ain = act[l];  // input activation of this layer
    float* pl = p64 + (size_t)(l & 1) * p64_set;
    // layer 0 reuses layer 2's set: its reduction on the side stream must be done
    if (l == 0)
      if (int e = stream_after(*ss, sd, st)) return e;
    int nparts = 0;
    if (int e = launch_wgrad64(gbuf[cur], ain, pl, L.nch64, B, H, W, status, st, &nparts)) return e;
    if (int e = stream_after(*ss, st, sd)) return e;
    prof_mark("dn_reduce", sd, false);
    k_reduce_wgrad64<<<(CH * CH * 9 + CH + 31) / 32, 256, 0, sd>>>(pl, nparts, grad_weights + o.w[l + 1],
                                                                     grad_weights + o.b[l + 1]);
    prof_mark("dn_reduce", sd, true);
    if (int e = launch_conv64(gbuf[cur], reinterpret_cast<__nv_bfloat16*>(w8 + L.wd[l]), nullptr, ain,
                              gbuf[cur ^ 1], 1, B, H, W, status, st))
      return e;
    cur ^= 1;
  }
  // first layer: weight gradient (side stream) and input gradient (+ residual)
  if (int e = stream_after(*ss, st, sd)) return e;
  prof_mark("dn_wgrad_small", sd, false);
  k_wgrad_l1<<<L.nch_small, 256, wl1_smem(W), sd>>>(B, H, W, gbuf[cur], xx, ps);
  prof_mark("dn_wgrad_small", sd, true);
  prof_mark("dn_reduce", sd, false);
  k_reduce_partials<<<(CH * 18 + CH + 31) / 32, 256, 0, sd>>>(ps, L.nch_small, kSmallOut, CH * 18,
                                                               grad_weights + o.w[0], CH, CH * 18,
                                                               grad_weights + o.b[0]);
  prof_mark("dn_reduce", sd, true);
  // first layer input gradient on the tensor cores: gx = gout + conv^T(g1) (flipped taps)
  if (int e = launch_conv64(gbuf[cur], reinterpret_cast<const __nv_bfloat16*>(w8 + L.ts[1]), nullptr, nullptr,
                            nullptr, 3, B, H, W, status, st, go, static_cast<float2*>(grad_x)))
    return e;
  // join
  if (int e = stream_after(*ss, sd, st)) return e;
  prof_count(8);  // every launch of the backward except the tensor-core kernels
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

}  // extern "C"

extern "C" int denoiser_get_status(void* ws, int B, int H, int W, void* stream, int* device_status) {
  if (!ws || !device_status) return SENSE_EINVAL_PTR;
  if (B <= 0 || H <= 0 || W <= 0) return SENSE_EINVAL_SHAPE;
  int* st = reinterpret_cast<int*>(static_cast<uint8_t*>(ws) + dn_layout(B, H, W).status);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  if (cudaMemcpyAsync(&v, st, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess || cudaMemsetAsync(st, 0, sizeof(int), s) != cudaSuccess)
    return SENSE_ECUDA;
  *device_status = v;
  return SENSE_OK;
}
