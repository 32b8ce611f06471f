// Internal declarations of the GB300 sparse-scoring library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include "gpusparse.h"

namespace gs {

constexpr int kBlock = GS_BLOCK;  // W = 32 postings per block (Sec. 3.2)

// One 32-posting block: 128 B of int32 doc ids, then 32 impacts.
__host__ __device__ constexpr int impact_bytes(int impact) {
  return impact == GS_IMPACT_F32 ? 4 : (impact == GS_IMPACT_U8 ? 1 : 2);
}
__host__ __device__ constexpr int block_bytes(int impact) { return 128 + 32 * impact_bytes(impact); }

// Workspace flag word bits (mirrors GS_FLAG_*).
constexpr uint32_t kFlagBadTerm = GS_FLAG_BAD_TERM;
constexpr uint32_t kFlagBadWeight = GS_FLAG_BAD_WEIGHT;
constexpr uint32_t kFlagCandOverflow = GS_FLAG_CAND_OVERFLOW;
constexpr uint32_t kFlagTimeout = GS_FLAG_TIMEOUT;
// flags that report invalid query data (the informational overflow bit aside)
constexpr uint32_t kDataFlags = GS_FLAG_BAD_TERM | GS_FLAG_BAD_WEIGHT | GS_FLAG_BAD_INDPTR;
// the status a synchronous call returns for a flag word
inline gs_status flags_status(uint32_t f) {
  if (f & kFlagTimeout) return GS_ERR_TIMEOUT;
  return (f & kDataFlags) ? GS_ERR_DATA : GS_OK;
}

}  // namespace gs

struct gs_index {
  int device = 0;
  int64_t N = 0;
  int32_t V = 0;
  int32_t impact = 0;
  int64_t nnz = 0;
  int64_t total_blocks = 0;
  int32_t blk_bytes = 0;
  int32_t tile_docs = 0;  // 0: no segment table
  int32_t num_tiles = 0;
  int32_t sms = 0;
  // device arrays
  uint8_t* blocks = nullptr;       // total_blocks * blk_bytes
  int64_t* term_block = nullptr;   // V + 1
  int32_t* term_len = nullptr;     // V
  float* max_score = nullptr;      // V
  float* max_abs = nullptr;        // V: largest |stored impact| of each list
  uint32_t* seg = nullptr;         // V * (num_tiles + 1)
  // dense head: the H longest lists as an [H][head_ld] impact matrix
  int32_t head_H = 0;
  int64_t head_ld = 0;
  int32_t* head_term = nullptr;    // H
  int32_t* head_slot = nullptr;    // V, -1 outside the head
  uint8_t* head_dense = nullptr;   // H * head_ld * impact_bytes
  // document-major copy for the doc-parallel kernel (optional)
  int64_t* dm_indptr = nullptr;    // N + 1
  int32_t* dm_terms = nullptr;     // nnz
  uint8_t* dm_impacts = nullptr;   // nnz * impact_bytes
  int64_t meta_bytes = 0;
  // host copies for planning
  std::vector<int64_t> h_term_block;
  std::vector<int32_t> h_term_len;
};

namespace gs {

// ---- order-preserving 32-bit keys: larger score <=> larger key ----
// float: -0 is folded onto +0 so that equal scores have equal keys.
__device__ __forceinline__ uint32_t score_key(float s) {
  uint32_t b = __float_as_uint(s);
  if (s == 0.0f) b = 0u;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ uint32_t score_key(int32_t s) { return (uint32_t)s ^ 0x80000000u; }
__device__ __forceinline__ float key_to_float(uint32_t k) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(b);
}
__device__ __forceinline__ int32_t key_to_int(uint32_t k) { return (int32_t)(k ^ 0x80000000u); }

// nearest-even integer of 51 * w (= w * 255 / 5) without FP64: the FMA
// residual of the float32 product decides a half-way float32 product.
__device__ __forceinline__ int32_t quant_u8(float w) {
  float p = __fmul_rn(51.0f, w);
  float e = __fmaf_rn(51.0f, w, -p);  // exact: 51 * w = p + e
  float r = rintf(p);
  if (fabsf(p - r) == 0.5f) {  // p is half-way between two integers
    if (e > 0.0f) r = ceilf(p);        // the exact product lies above p
    else if (e < 0.0f) r = floorf(p);  // ... below p; e == 0: a true tie, even
  }
  if (!(r >= 0.0f)) r = 0.0f;
  if (r > 255.0f) r = 255.0f;
  return (int32_t)r;
}

// ---- workspace carving ----
struct Carver {
  uint8_t* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<uint8_t*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t size() const { return (off + 255) & ~size_t(255); }
};

// error helpers
void set_cuda_error(cudaError_t e);
int device_sm_count(int device);
// launch accounting and stage events
void count_launches(int n);
void record_stage(const gs_search_opts* opts, int i, cudaStream_t s);

}  // namespace gs

#define GS_CUDA_TRY(expr)                 \
  do {                                    \
    cudaError_t _e = (expr);              \
    if (_e != cudaSuccess) {              \
      gs::set_cuda_error(_e);             \
      return GS_ERR_CUDA;                 \
    }                                     \
  } while (0)

// checks the launch(es) just made and counts n kernels
#define GS_LAUNCH_CHECK_N(n)                \
  do {                                      \
    cudaError_t _e = cudaGetLastError();    \
    if (_e != cudaSuccess) {                \
      gs::set_cuda_error(_e);               \
      return GS_ERR_CUDA;                   \
    }                                       \
    gs::count_launches(n);                  \
  } while (0)
#define GS_LAUNCH_CHECK() GS_LAUNCH_CHECK_N(1)
