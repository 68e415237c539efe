// Side streams of the library (see plan.cuh): three non-blocking streams per device and one event
// used for fork and join (each record is waited on at once, so one event serves every edge).
#include <mutex>

#include "plan.cuh"

namespace {
constexpr int kDevs = 64;
SideSet g_sets[kDevs];
bool g_ready[kDevs] = {};
std::mutex g_mu;
}  // namespace

int side_set(SideSet** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) return SENSE_ECUDA;
  std::lock_guard<std::mutex> l(g_mu);
  SideSet& ss = g_sets[dev];
  if (!g_ready[dev]) {
    int made = 0;  // streams created so far
    while (made < kSideStreams && cudaStreamCreateWithFlags(&ss.s[made], cudaStreamNonBlocking) == cudaSuccess)
      ++made;
    const bool ok = made == kSideStreams && cudaEventCreateWithFlags(&ss.ev, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {  // release what was made; the next call tries again
      for (int i = 0; i < made; ++i) cudaStreamDestroy(ss.s[i]);
      return SENSE_ECUDA;
    }
    g_ready[dev] = true;
  }
  *out = &ss;
  return SENSE_OK;
}

int stream_after(const SideSet& ss, cudaStream_t from, cudaStream_t to) {
  std::lock_guard<std::mutex> l(g_mu);  // record and wait as one step for every host thread
  if (cudaEventRecord(ss.ev, from) != cudaSuccess || cudaStreamWaitEvent(to, ss.ev, 0) != cudaSuccess)
    return SENSE_ECUDA;
  return SENSE_OK;
}

extern "C" int sense_streams_join(void* stream) {
  SideSet* ss = nullptr;
  if (int e = side_set(&ss)) return e;
  const cudaStream_t to = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < kSideStreams; ++i)
    if (int e = stream_after(*ss, ss->s[i], to)) return e;
  return SENSE_OK;
}
