// Small C-ABI helpers: status strings, CUDA error capture, version.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <unordered_map>

#include "gs_internal.cuh"

namespace gs {

static thread_local cudaError_t t_last_cuda = cudaSuccess;

void set_cuda_error(cudaError_t e) { t_last_cuda = e; }

static std::atomic<int64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void record_stage(const gs_search_opts* opts, int i, cudaStream_t s) {
  if (opts && opts->stage_events && i >= 0 && i < GS_NUM_STAGE_EVENTS && opts->stage_events[i])
    cudaEventRecord(static_cast<cudaEvent_t>(opts->stage_events[i]), s);
}

int device_sm_count(int device) {
  static std::mutex mu;
  static std::unordered_map<int, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(device);
  if (it != cache.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) sms = 1;
  cache[device] = sms;
  return sms;
}

}  // namespace gs

extern "C" const char* gs_status_str(gs_status s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_OUT_OF_MEMORY: return "out of device memory";
    case GS_ERR_CUDA: return "CUDA runtime error";
    case GS_ERR_UNSUPPORTED: return "unsupported";
    case GS_ERR_DATA: return "invalid document data";
    case GS_ERR_TIMEOUT: return "device wait timed out";
    case GS_ERR_WORKSPACE: return "workspace too small";
  }
  return "unknown status";
}

extern "C" const char* gs_last_cuda_error(void) { return cudaGetErrorString(gs::t_last_cuda); }

extern "C" int32_t gs_version(void) { return 100; }

extern "C" int64_t gs_kernel_launches(void) { return gs::g_launches.load(); }
