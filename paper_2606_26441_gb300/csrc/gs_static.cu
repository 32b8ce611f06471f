// gs_search_static: exact top-k search for callers that cannot allocate
// device memory.  Its scratch lives in one fixed-size array of device memory
// that the library declares at file scope; every GPU that loads the library
// holds that array (GS_STATIC_SCRATCH_BYTES) until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "gs_internal.cuh"

namespace {

__device__ __align__(256) uint8_t g_static_scratch[GS_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device, with that device current.
gs_status scratch_for_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    gs::set_cuda_error(e);
    return GS_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return GS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      gs::set_cuda_error(e);
      return GS_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GS_OK;
}

}  // namespace

extern "C" gs_status gs_search_static(const gs_index* index, const int32_t* q_indptr, const int32_t* q_terms,
                                      const float* q_w, int32_t batch, int64_t q_nnz, int32_t k, int32_t* out_ids,
                                      void* out_scores, const gs_search_opts* opts, gs_stream_t stream) {
  size_t need = 0;
  gs_status st = gs_search_workspace_size(index, batch, q_nnz, k, opts, 0, &need);
  if (st != GS_OK) return st;
  if (need > (size_t)GS_STATIC_SCRATCH_BYTES) return GS_ERR_WORKSPACE;
  void* scratch = nullptr;
  st = scratch_for_current_device(&scratch);
  if (st != GS_OK) return st;
  // gs_search clears every part of its scratch it relies on being zero, so the
  // previous call's leftovers do no harm
  return gs_search(index, q_indptr, q_terms, q_w, batch, q_nnz, k, out_ids, out_scores, scratch,
                   (size_t)GS_STATIC_SCRATCH_BYTES, opts, stream);
}

extern "C" gs_status gs_search_static_flags(gs_stream_t stream, uint32_t* flags) {
  if (!flags) return GS_ERR_INVALID_ARG;
  void* scratch = nullptr;
  gs_status st = scratch_for_current_device(&scratch);
  if (st != GS_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(flags, scratch, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    gs::set_cuda_error(e);
    return GS_ERR_CUDA;
  }
  return GS_OK;
}
