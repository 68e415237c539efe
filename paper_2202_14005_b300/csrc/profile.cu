// Process-wide launch accounting and optional CUDA-event timing per kernel
// class (the fused normal operator, the tensor-core convolution, the weight
// gradients, ...).  Events are recorded on the stream each kernel is launched
// on, immediately before and after the launch.
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "plan.cuh"

namespace {

struct Rec {
  std::vector<cudaEvent_t> ev;  // start/stop pairs
  int used = 0;
};

std::mutex g_mu;
int g_on = 0;
long long g_launches = 0;
std::map<std::string, Rec> g_recs;

}  // namespace

void prof_count(int n) {
  std::lock_guard<std::mutex> l(g_mu);
  g_launches += n;
}

void prof_mark(const char* name, cudaStream_t s, bool stop) {
  std::lock_guard<std::mutex> l(g_mu);
  if (!g_on) return;
  Rec& r = g_recs[name];
  const size_t need = 2 * (size_t)r.used + 2;
  while (r.ev.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    r.ev.push_back(e);
  }
  cudaEventRecord(r.ev[2 * (size_t)r.used + (stop ? 1 : 0)], s);
  if (stop) ++r.used;
}

extern "C" {

int sense_profile_enable(int enable) {
  std::lock_guard<std::mutex> l(g_mu);
  g_on = enable ? 1 : 0;
  return SENSE_OK;
}

int sense_profile_read(const char* name, double* ms, int* launches) {
  if (!name) return SENSE_EINVAL_PTR;
  std::lock_guard<std::mutex> l(g_mu);
  double t = 0.0;
  int n = 0;
  auto it = g_recs.find(name);
  if (it != g_recs.end()) {
    Rec& r = it->second;
    for (int i = 0; i < r.used; ++i) {
      if (cudaEventSynchronize(r.ev[2 * (size_t)i + 1]) != cudaSuccess) return SENSE_ECUDA;
      float f = 0.f;
      if (cudaEventElapsedTime(&f, r.ev[2 * (size_t)i], r.ev[2 * (size_t)i + 1]) != cudaSuccess)
        return SENSE_ECUDA;
      t += f;
    }
    n = r.used;
    r.used = 0;
  }
  if (ms) *ms = t;
  if (launches) *launches = n;
  return SENSE_OK;
}

// FP32 FMA throughput probe: every thread runs 8 independent FMA chains of `iters` steps in
// registers (no memory traffic until one store per thread), so the achieved rate is the FP32
// pipe's peak at the clock the GPU runs.  2 * 8 * iters * 256 FLOP per thread-block.
__global__ void __launch_bounds__(256) k_fma_probe(int iters, float seed, float* sink) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + 1e-3f * (threadIdx.x + 37 * k);
  const float m = 0.999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 12345.678f) sink[blockIdx.x] = s;  // keeps the chains live; practically never taken
}

int sense_fma_probe(int blocks, int iters, float* sink, void* stream) {
  if (blocks <= 0 || iters <= 0) return SENSE_EINVAL_ARG;
  if (!sink) return SENSE_EINVAL_PTR;
  k_fma_probe<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(iters, 1.0f, sink);
  prof_count(1);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

long long sense_kernel_launches(int reset) {
  std::lock_guard<std::mutex> l(g_mu);
  const long long v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

}  // extern "C"
