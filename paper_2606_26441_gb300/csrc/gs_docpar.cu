// Doc-parallel scoring (Sec. 5.3) and the merge of per-shard top-k lists.
//
// Doc-parallel: the queries of the batch become a dense term-major matrix
// Qd[V][Bp] (Bp = batch rounded up to 8); one thread per document walks the
// document's own terms (the index's document-major copy) and, for 8 queries
// at a time, adds x_d(t) * Qd[t][q] in registers, then writes the 8 scores.
// No atomics: every (query, document) score has one owner.  It reads every
// posting once per 8 queries, the work-inefficient side of the paper's
// work-versus-bandwidth tradeoff; the dense rows then go through the dense
// top-k.
#include <cuda_runtime.h>

#include <algorithm>

#include "gs_docpar.cuh"
#include "gs_topk.cuh"

namespace gs {

// the shard tables travel by value as a kernel parameter: nothing is allocated
struct MergeTables {
  const int32_t* ids[GS_MAX_SHARDS];
  const void* sc[GS_MAX_SHARDS];
  int64_t off[GS_MAX_SHARDS];
};

template <typename ST>
__global__ void __launch_bounds__(1024) merge_topk_kernel(const MergeTables T, int S, int k_in, int k,
                                                          int32_t* __restrict__ out_ids, ST* __restrict__ out_scores);

namespace {

struct DpPlan {
  uint32_t* qd;  // [V][Bp] float or int
  uint32_t* rows;
  int64_t ld;
  int Bp;
};

DpPlan carve_dp(void* ws, const gs_index* ix, int B, size_t* bytes) {
  Carver c(ws);
  DpPlan p{};
  p.Bp = (B + 7) / 8 * 8;
  p.qd = c.take<uint32_t>((size_t)ix->V * p.Bp);
  p.ld = (ix->N + 31) / 32 * 32;
  p.rows = c.take<uint32_t>((size_t)B * p.ld);
  *bytes = c.size();
  return p;
}

__global__ void dp_zero_kernel(uint4* __restrict__ p, int64_t n4) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) p[i] = make_uint4(0, 0, 0, 0);
}

// dense term-major query matrix; repeated terms add up; bad entries are skipped
__global__ void dp_query_kernel(const int32_t* __restrict__ q_indptr, const int32_t* __restrict__ q_terms,
                                const float* __restrict__ q_w, int32_t B, int64_t q_nnz, int32_t V, int impact,
                                int Bp, uint32_t* __restrict__ qd, uint32_t* flags) {
  uint32_t fl = 0;
  const int64_t used = min((int64_t)max(q_indptr[B], 0), q_nnz);
  if (blockIdx.x == 0 && threadIdx.x == 0 && (q_indptr[0] != 0 || q_indptr[B] > q_nnz)) fl |= GS_FLAG_BAD_INDPTR;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < used; p += stride) {
    int lo = 0, hi = B + 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (q_indptr[mid] <= (int32_t)p) lo = mid + 1; else hi = mid;
    }
    const int q = lo - 1;
    const int32_t t = q_terms[p];
    const float w = q_w[p];
    if (t < 0 || t >= V) { fl |= kFlagBadTerm; continue; }
    if (!isfinite(w)) { fl |= kFlagBadWeight; continue; }
    if (q < 0 || q >= B) continue;
    uint32_t* cell = qd + (int64_t)t * Bp + q;
    if (impact == GS_IMPACT_U8) atomicAdd(reinterpret_cast<int32_t*>(cell), quant_u8(w));
    else atomicAdd(reinterpret_cast<float*>(cell), w);
  }
  if (fl) atomicOr(flags, fl);
}

template <int IMPACT>
__device__ __forceinline__ float dm_impact(const uint8_t* imp, int64_t p) {
  if (IMPACT == GS_IMPACT_F32) return __ldg(reinterpret_cast<const float*>(imp) + p);
  if (IMPACT == GS_IMPACT_F16) return __half2float(__ldg(reinterpret_cast<const __half*>(imp) + p));
  if (IMPACT == GS_IMPACT_BF16) return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(imp) + p));
  return (float)__ldg(imp + p);
}

template <int IMPACT>
__global__ void __launch_bounds__(256) dp_score_kernel(const int64_t* __restrict__ dm_indptr,
                                                       const int32_t* __restrict__ dm_terms,
                                                       const uint8_t* __restrict__ dm_imp, int64_t N, int32_t B,
                                                       int Bp, const uint32_t* __restrict__ qd, int64_t ld,
                                                       uint32_t* __restrict__ rows) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += stride) {
    const int64_t a = dm_indptr[d], b = dm_indptr[d + 1];
    for (int q0 = 0; q0 < B; q0 += 8) {
      if (IMPACT == GS_IMPACT_U8) {
        int32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t p = a; p < b; ++p) {
          const int32_t x = (int32_t)__ldg(dm_imp + p);
          const uint4* w4 = reinterpret_cast<const uint4*>(qd + (int64_t)__ldg(dm_terms + p) * Bp + q0);
          const uint4 u0 = __ldg(w4), u1 = __ldg(w4 + 1);
          acc[0] += (int32_t)u0.x * x; acc[1] += (int32_t)u0.y * x; acc[2] += (int32_t)u0.z * x;
          acc[3] += (int32_t)u0.w * x; acc[4] += (int32_t)u1.x * x; acc[5] += (int32_t)u1.y * x;
          acc[6] += (int32_t)u1.z * x; acc[7] += (int32_t)u1.w * x;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (q0 + j < B) rows[(int64_t)(q0 + j) * ld + d] = (uint32_t)acc[j];
      } else {
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int64_t p = a; p < b; ++p) {
          const float x = dm_impact<IMPACT>(dm_imp, p);
          const float4* w4 = reinterpret_cast<const float4*>(qd + (int64_t)__ldg(dm_terms + p) * Bp + q0);
          const float4 u0 = __ldg(w4), u1 = __ldg(w4 + 1);
          acc[0] = fmaf(u0.x, x, acc[0]); acc[1] = fmaf(u0.y, x, acc[1]); acc[2] = fmaf(u0.z, x, acc[2]);
          acc[3] = fmaf(u0.w, x, acc[3]); acc[4] = fmaf(u1.x, x, acc[4]); acc[5] = fmaf(u1.y, x, acc[5]);
          acc[6] = fmaf(u1.z, x, acc[6]); acc[7] = fmaf(u1.w, x, acc[7]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (q0 + j < B) rows[(int64_t)(q0 + j) * ld + d] = __float_as_uint(acc[j]);
      }
    }
  }
}

}  // namespace

template <typename ST>
__global__ void __launch_bounds__(1024) merge_topk_kernel(const MergeTables T, int S, int k_in, int k,
                                                          int32_t* __restrict__ out_ids, ST* __restrict__ out_scores) {
  __shared__ uint32_t hist[2048];
  __shared__ uint32_t ck[GS_MAX_K];
  __shared__ int32_t cid[GS_MAX_K];
  __shared__ int warp_buf[32];
  __shared__ uint32_t s_digit;
  __shared__ int s_need, s_fill;
  const int q = blockIdx.x;
  auto get = [&](int64_t i) -> uint2 {
    const int s = (int)(i / k_in), j = (int)(i - (int64_t)s * k_in);
    const int64_t at = (int64_t)q * k_in + j;
    const ST v = reinterpret_cast<const ST*>(T.sc[s])[at];
    return make_uint2(score_key(v), (uint32_t)(T.ids[s][at] + T.off[s]));
  };
  select_topk_candidates(get, (int64_t)S * k_in, k, hist, warp_buf, &s_digit, &s_need, &s_fill, ck, cid);
  int n_pad = 1;
  while (n_pad < k) n_pad <<= 1;
  for (int i = k + threadIdx.x; i < n_pad; i += blockDim.x) {
    ck[i] = 0u;
    cid[i] = 0x7fffffff;
  }
  bitonic_sort_desc(ck, cid, n_pad);
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    out_ids[(int64_t)q * k + j] = cid[j];
    out_scores[(int64_t)q * k + j] = key_to_score<ST>(ck[j]);
  }
}

namespace {

template <int IMPACT>
void launch_dp(const gs_index* ix, int B, const DpPlan& p, cudaStream_t s) {
  const int grid = std::max(1, ix->sms) * 8;
  dp_score_kernel<IMPACT><<<grid, 256, 0, s>>>(ix->dm_indptr, ix->dm_terms, ix->dm_impacts, ix->N, B, p.Bp, p.qd, p.ld,
                                               p.rows);
}

}  // namespace

}  // namespace gs

namespace gs {

gs_status dp_workspace_bytes(const gs_index* ix, int32_t B, size_t* bytes) {
  if (!ix->dm_indptr) return GS_ERR_UNSUPPORTED;
  carve_dp(nullptr, ix, B, bytes);
  return GS_OK;
}

gs_status dp_search(const gs_index* ix, const int32_t* q_indptr, const int32_t* q_terms, const float* q_w, int32_t B,
                    int64_t q_nnz, int32_t k, int32_t* out_ids, void* out_scores, void* ws, size_t ws_bytes,
                    uint32_t* flags, const gs_search_opts* opts, cudaStream_t s) {
  if (!ix->dm_indptr) return GS_ERR_UNSUPPORTED;
  size_t need = 0;
  DpPlan p = carve_dp(ws, ix, B, &need);
  if (need > ws_bytes) return GS_ERR_WORKSPACE;
  record_stage(opts, 0, s);
  const int64_t n4 = (int64_t)ix->V * p.Bp / 4;
  dp_zero_kernel<<<std::max(1, ix->sms) * 4, 256, 0, s>>>(reinterpret_cast<uint4*>(p.qd), n4);
  GS_LAUNCH_CHECK();
  dp_query_kernel<<<(int)std::min<int64_t>((q_nnz + 255) / 256 + 1, 4096), 256, 0, s>>>(
      q_indptr, q_terms, q_w, B, q_nnz, ix->V, ix->impact, p.Bp, p.qd, flags);
  GS_LAUNCH_CHECK();
  record_stage(opts, 1, s);
  record_stage(opts, 2, s);
  record_stage(opts, 3, s);
  switch (ix->impact) {
    case GS_IMPACT_F32: launch_dp<GS_IMPACT_F32>(ix, B, p, s); break;
    case GS_IMPACT_F16: launch_dp<GS_IMPACT_F16>(ix, B, p, s); break;
    case GS_IMPACT_BF16: launch_dp<GS_IMPACT_BF16>(ix, B, p, s); break;
    default: launch_dp<GS_IMPACT_U8>(ix, B, p, s); break;
  }
  GS_LAUNCH_CHECK();
  record_stage(opts, 4, s);
  if (ix->impact == GS_IMPACT_U8)
    topk_dense_rows_kernel<int32_t><<<B, kTopkThreads, 0, s>>>(reinterpret_cast<const int32_t*>(p.rows), p.ld, ix->N,
                                                              k, out_ids, static_cast<int32_t*>(out_scores), nullptr);
  else
    topk_dense_rows_kernel<float><<<B, kTopkThreads, 0, s>>>(reinterpret_cast<const float*>(p.rows), p.ld, ix->N, k,
                                                            out_ids, static_cast<float*>(out_scores), nullptr);
  GS_LAUNCH_CHECK();
  record_stage(opts, 5, s);
  return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_merge_topk(const int32_t* const* shard_ids, const void* const* shard_scores,
                                   const int64_t* doc_offset, int32_t n_shards, int32_t batch, int32_t k_in, int32_t k,
                                   int32_t score_is_int, int32_t* out_ids, void* out_scores, gs_stream_t stream) {
  if (!shard_ids || !shard_scores || !doc_offset || n_shards < 1 || n_shards > GS_MAX_SHARDS || batch < 1 ||
      k_in < 1 || k < 1 || (int64_t)k > (int64_t)n_shards * k_in || !out_ids || !out_scores)
    return GS_ERR_INVALID_ARG;
  if (k > GS_MAX_K) return GS_ERR_UNSUPPORTED;
  for (int s = 0; s < n_shards; ++s)
    if (!shard_ids[s] || !shard_scores[s] || doc_offset[s] < 0) return GS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MergeTables T{};
  for (int i = 0; i < n_shards; ++i) {
    T.ids[i] = shard_ids[i];
    T.sc[i] = shard_scores[i];
    T.off[i] = doc_offset[i];
  }
  if (score_is_int)
    merge_topk_kernel<int32_t><<<batch, 1024, 0, s>>>(T, n_shards, k_in, k, out_ids, static_cast<int32_t*>(out_scores));
  else
    merge_topk_kernel<float><<<batch, 1024, 0, s>>>(T, n_shards, k_in, k, out_ids, static_cast<float*>(out_scores));
  GS_LAUNCH_CHECK();
  return GS_OK;
}
