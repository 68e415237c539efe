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

// Device address of g_noalloc_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return SENSE_EINVAL_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SENSE_ECUDA;
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return SENSE_OK;
}

// One warp per image row: FP32 products of two complex values per step, summed
// per lane, then an FP64 warp sum; the last CTA reduces the per-row partials of
// each slice in row order and (count == 1) the slices in slice order.
__global__ void __launch_bounds__(kWarps * 32)
k_dot_noalloc(int B, int H, int W, const float2* a, const float2* b, const float2* c,
              double* out, int count, unsigned* counter, double* part) {
  const int row = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row < B * H) {
    const size_t off = (size_t)row * W / 2;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    const float4* c4 = reinterpret_cast<const float4*>(c);
    float s = 0.f;
    for (int i = lane; i < W / 2; i += 32) {
      const float4 u = a4[off + i];
      float4 v = b ? b4[off + i] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (c) {
        const float4 w = c4[off + i];
        v.x -= w.x; v.y -= w.y; v.z -= w.z; v.w -= w.w;
      }
      s = fmaf(u.x, v.x, fmaf(u.y, v.y, fmaf(u.z, v.z, fmaf(u.w, v.w, s))));
    }
    const double d = warp_sum_d((double)s);
    if (lane == 0) part[row] = d;
  }
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    double total = 0.0;
    for (int bb = 0; bb < B; ++bb) {
      double t = 0.0;
      for (int i = lane; i < H; i += 32) t += __ldcg(part + (size_t)bb * H + i);
      t = warp_sum_d(t);
      if (count == B) {
        if (lane == 0) out[bb] = t;
      } else {
        total += t;
      }
    }
    if (count != B && lane == 0) out[0] = total;
    if (lane == 0) *counter = 0u;
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
  void* base = nullptr;
  if (int e = scratch_address(dev, &base)) return e;
  unsigned* counter = static_cast<unsigned*>(base);
  double* part = reinterpret_cast<double*>(static_cast<char*>(base) + kCounterBytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the counter must start at zero; the partials are all overwritten
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), st) != cudaSuccess) return SENSE_ECUDA;
  const int grid = (B * H + kWarps - 1) / kWarps;
  k_dot_noalloc<<<grid, kWarps * 32, 0, st>>>(B, H, W, static_cast<const float2*>(a),
                                              static_cast<const float2*>(b),
                                              static_cast<const float2*>(c), out, out_count,
                                              counter, part);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}
