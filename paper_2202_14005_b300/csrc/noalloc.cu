// sense_dot_re_noalloc: the per-slice inner product Re<a, b - c> of the CG
// backward (the lambda gradient), for callers that may not allocate device
// memory.  Its scratch (per-row FP64 partials and the last-block counter) lives
// in a fixed file-scope device array instead of a workspace.  The paper has no
// counterpart; see include/sense.h for the contract.
#include <cstdint>
#include <mutex>

#include "plan.cuh"

namespace {

constexpr int kWarps = 8;
constexpr size_t kCounterBytes = 256;  // counter at the front, partials after it

// Scratch shared by every call in this process, on every device that loads the
// library (each holds its own copy until the process exits).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SENSE_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device.  It is looked up on a device's
// first call (the set-up) and looked up again by every later call made outside
// stream capture, so an address that moved with a device reset is never used
// by such a call; a call under capture uses the last address found.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

int scratch_address(int device, cudaStream_t st, void** out) {
  if (device < 0 || device >= kMaxDevices) return SENSE_EINVAL_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SENSE_ECUDA;
  if (!g_addr[device] || cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SENSE_ECUDA;
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return SENSE_OK;
}

// The row split and the order of every summation are those of the workspace
// kernel behind cg_dc_solve_backward's lambda gradient, so both give the same
// bits: two warps per image row (four rows per CTA), each thread summing the
// FP32 products of two complex values per step, an FP64 sum per warp, the two
// warp sums of a row added in warp order; the last CTA reduces each slice's
// row partials with the same lane-strided FP64 sum and, for count == 1, adds
// the slice totals in slice order.
constexpr int kRowsPerCta = kWarps / 2;

__global__ void __launch_bounds__(kWarps * 32)
k_dot_noalloc(int B, int H, int W, const float2* a, const float2* b, const float2* c,
              double* out, int count, unsigned* counter, double* part) {
  const int row = blockIdx.x * kRowsPerCta + (threadIdx.x >> 6);
  const int lt = threadIdx.x & 63;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool rv = row < B * H;
  float s = 0.f;
  if (rv) {
    const size_t off = (size_t)row * W / 2;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    const float4* c4 = reinterpret_cast<const float4*>(c);
    for (int i = lt; i < W / 2; i += 64) {
      const float4 u = a4[off + i];
      float4 v = b ? b4[off + i] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (c) {
        const float4 w = c4[off + i];
        v.x -= w.x; v.y -= w.y; v.z -= w.z; v.w -= w.w;
      }
      s += fmaf(u.x, v.x, fmaf(u.y, v.y, fmaf(u.z, v.z, u.w * v.w)));
    }
  }
  __shared__ double s_w[kWarps];
  const double d = warp_sum_d((double)s);
  if (lane == 0) s_w[warp] = d;
  __syncthreads();
  if (rv && (threadIdx.x & 63) == 0) part[row] = s_w[warp] + s_w[warp + 1];

  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ double s_slice[kWarps];
  double total = 0.0;  // thread 0: slice totals added in slice order
  for (int b0 = 0; b0 < B; b0 += kWarps) {
    const int bb = b0 + warp;
    if (bb < B) {
      double t = lane_strided_sum(part + (size_t)bb * H, H, lane);
      t = warp_sum_d(t);
      if (lane == 0) {
        if (count == B) out[bb] = t;
        else s_slice[warp] = t;
      }
    }
    __syncthreads();
    if (count != B && threadIdx.x == 0)
      for (int k = 0; k < kWarps && b0 + k < B; ++k) total += s_slice[k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (count != B) out[0] = total;
    *counter = 0u;
  }
}

bool aligned(const void* p, unsigned m) { return ((uintptr_t)p & (m - 1)) == 0; }

}  // namespace

extern "C" int sense_dot_re_noalloc(int B, int H, int W, const void* a, const void* b,
                                    const void* c, double* out, int out_count, void* stream) {
  if (B <= 0 || H <= 0 || W <= 0 || (W & 1)) return SENSE_EINVAL_SHAPE;
  if (!a || !out || !aligned(a, 16) || (b && !aligned(b, 16)) || (c && !aligned(c, 16)) ||
      !aligned(out, 8))
    return SENSE_EINVAL_PTR;
  if (out_count != 1 && out_count != B) return SENSE_EINVAL_ARG;
  if ((size_t)B * H > SENSE_NOALLOC_MAX_ROWS) return SENSE_ETOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SENSE_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* base = nullptr;
  if (int e = scratch_address(dev, st, &base)) return e;
  unsigned* counter = static_cast<unsigned*>(base);
  double* part = reinterpret_cast<double*>(static_cast<char*>(base) + kCounterBytes);
  // the counter must start at zero; the partials are all overwritten
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), st) != cudaSuccess) return SENSE_ECUDA;
  const int grid = (B * H + kRowsPerCta - 1) / kRowsPerCta;
  k_dot_noalloc<<<grid, kWarps * 32, 0, st>>>(B, H, W, static_cast<const float2*>(a),
                                              static_cast<const float2*>(b),
                                              static_cast<const float2*>(c), out, out_count,
                                              counter, part);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}
