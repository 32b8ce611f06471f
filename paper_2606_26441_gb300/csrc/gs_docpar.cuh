// Doc-parallel scoring path (declarations).
#pragma once

#include "gs_internal.cuh"

namespace gs {

gs_status dp_workspace_bytes(const gs_index* ix, int32_t B, size_t* bytes);

gs_status dp_search(const gs_index* ix, const int32_t* q_indptr, const int32_t* q_terms, const float* q_w, int32_t B,
                    int64_t q_nnz, int32_t k, int32_t* out_ids, void* out_scores, void* ws, size_t ws_bytes,
                    uint32_t* flags, const gs_search_opts* opts, cudaStream_t s);

}  // namespace gs
