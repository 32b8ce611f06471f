// Doc-tiled scoring path (declarations).
#pragma once

#include "gs_internal.cuh"

namespace gs {

// Workspace bytes of the doc-tiled path (placed after the term-parallel region).
gs_status dt_workspace_bytes(const gs_index* ix, int32_t B, int64_t q_nnz, int32_t k, const gs_search_opts* opts,
                             size_t* bytes);

// Resolved doc-tiled plan (G, T, R, ...) for gs_search_plan.
gs_status dt_plan_info(const gs_index* ix, int32_t B, int32_t k, const gs_search_opts* opts, gs_plan_info* out);

// Runs the doc-tiled search on `s`; flags: the workspace flag word.
gs_status dt_search(const gs_index* ix, const int32_t* q_indptr, const int32_t* q_terms, const float* q_w,
                    int32_t B, int64_t q_nnz, int32_t k, int32_t* out_ids, void* out_scores, void* ws,
                    size_t ws_bytes, uint32_t* flags, const gs_search_opts* opts, cudaStream_t s);

// Raises the doc-tiled kernels' dynamic shared-memory ceilings for the index's
// impact type on the current device (every head kind) and records the recovery
// kernel's occupancy; idempotent.
gs_status dt_prepare_device(const gs_index* ix);

// Exact top-k of B dense score rows (row q at rows + q * ld, N scores, float
// or int32 on the uint8 path) by a sampled threshold and one candidate pass;
// rows whose candidates overflow are selected again over the whole row.  The
// workspace is separate from the rows; flags: a flag word.
gs_status dense_topk_workspace_bytes(const gs_index* ix, int32_t B, int32_t k, size_t* bytes);
gs_status dense_topk(const gs_index* ix, const void* rows, int64_t ld, int32_t B, int32_t k, int32_t* out_ids,
                     void* out_scores, void* ws, size_t ws_bytes, uint32_t* flags, cudaStream_t s);

}  // namespace gs
