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

// Query order of a doc-tiled batch (gs_order.cu): whether the batch is
// regrouped (groups of at least 8 queries and two groups or more; by default
// only where a cost model predicts a gain, see gs_search_opts.query_order),
// the device set-up index builds call, and the launch:
// the regrouped query CSR goes to o_indptr [B + 1], o_terms / o_w [q_nnz], and
// perm [B] holds the caller's query at each position.  head_slot: the dense
// head's term slots when the search uses the head (its terms do not count),
// else NULL.
bool dt_order_used(int32_t B, int G, int64_t N, const gs_search_opts* opts);
// Copies the order of the last regrouped search on this doc-tiled workspace
// region (GS_ERR_UNSUPPORTED when these arguments do not regroup).
gs_status dt_order_of(const gs_index* ix, int32_t B, int64_t q_nnz, int32_t k, const gs_search_opts* opts,
                      const void* ws, size_t ws_bytes, int32_t* out_perm, cudaStream_t s);
gs_status dt_order_prepare_device();
gs_status dt_order(const gs_index* ix, const int32_t* q_indptr, const int32_t* q_terms, const float* q_w, int32_t B,
                   int32_t q_nnz, int G, const int32_t* head_slot, int32_t* o_indptr, int32_t* o_terms, float* o_w,
                   int32_t* perm, cudaStream_t s);

// Exact top-k of B dense score rows (row q at rows + q * ld, N scores, float
// or int32 on the uint8 path) by a sampled threshold and one candidate pass;
// rows whose candidates overflow are selected again over the whole row.  The
// workspace is separate from the rows; flags: a flag word.
gs_status dense_topk_workspace_bytes(const gs_index* ix, int32_t B, int32_t k, size_t* bytes);
gs_status dense_topk(const gs_index* ix, const void* rows, int64_t ld, int32_t B, int32_t k, int32_t* out_ids,
                     void* out_scores, void* ws, size_t ws_bytes, uint32_t* flags, cudaStream_t s);

}  // namespace gs
