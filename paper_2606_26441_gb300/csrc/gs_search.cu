// Search entry points, workspace planning and the term-parallel scatter-add
// (Sec. 4.2 and the fused kernel of Sec. 5.2, re-designed for sm_103a):
//   prep   : one CTA validates the query CSR and turns every (query, term)
//            pair into ceil(blocks(t) / chunk) work items (exclusive prefix);
//   zero   : the [B x ld] score rows;
//   scatter: a persistent grid of warps takes work items in query-major order
//            (so the rows in flight stay L2-resident); each warp reads 4
//            posting blocks per step with 128-bit loads (8 lanes per block,
//            4 postings per lane) and adds w * x into the row with global
//            reductions; padding (doc -1) is skipped;
//   top-k  : gs_topk.cuh over the rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "gs_docpar.cuh"
#include "gs_doctiled.cuh"
#include "gs_internal.cuh"
#include "gs_topk.cuh"

namespace gs {
namespace {

constexpr int kPrepThreads = 1024;
constexpr int kDefaultChunkBlocks = 32;  // 1024 postings per work item (Sec. 5.2 tunes BLOCK_PL)

struct Header {
  uint32_t flags;
  uint32_t pad0;
  int64_t total_chunks;
  uint32_t reserved[60];
};

__device__ __forceinline__ int64_t upper_bound_i64(const int64_t* a, int64_t n, int64_t v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int upper_bound_i32(const int32_t* a, int n, int32_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One CTA: per (query, term) pair its query row, validated term and weight,
// and the exclusive prefix of work items.  Bad pairs get no work and raise a
// flag (the term is skipped, as the contract states).
__global__ void __launch_bounds__(kPrepThreads) tp_prep_kernel(
    const int32_t* __restrict__ q_indptr, const int32_t* __restrict__ q_terms, const float* __restrict__ q_w,
    int32_t B, int64_t q_nnz, int32_t V, int impact, const int64_t* __restrict__ term_block, int chunk_blocks,
    int32_t* __restrict__ pair_q, int32_t* __restrict__ pair_t, float* __restrict__ pair_wf,
    int32_t* __restrict__ pair_wi, int64_t* __restrict__ pair_chunk, Header* hdr) {
  __shared__ int warp_buf[32];
  __shared__ int64_t s_carry;
  __shared__ int64_t s_wsum[32];
  if (threadIdx.x == 0) s_carry = 0;
  uint32_t flags = 0;
  // indptr sanity (device data): monotone, ends at q_nnz
  for (int q = threadIdx.x; q < B; q += blockDim.x) {
    if (q_indptr[q + 1] < q_indptr[q]) flags |= GS_FLAG_BAD_INDPTR;
  }
  if (threadIdx.x == 0 && (q_indptr[0] != 0 || (int64_t)q_indptr[B] > q_nnz || q_indptr[B] < 0))
    flags |= GS_FLAG_BAD_INDPTR;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // entries past q_indptr[B] are unused capacity
  const int64_t n_used = min((int64_t)max(q_indptr[B], 0), q_nnz);
  for (int64_t base = 0; base < q_nnz; base += blockDim.x) {
    const int64_t p = base + threadIdx.x;
    int64_t nch = 0;
    if (p < q_nnz) {
      pair_q[p] = 0;
      pair_t[p] = 0;
    }
    if (p < n_used) {
      const int q = upper_bound_i32(q_indptr, B + 1, (int32_t)p) - 1;
      const int32_t t = q_terms[p];
      const float w = q_w[p];
      const bool bad_t = (t < 0 || t >= V);
      const bool bad_w = !isfinite(w);
      if (bad_t) flags |= kFlagBadTerm;
      if (bad_w) flags |= kFlagBadWeight;
      pair_q[p] = min(max(q, 0), B - 1);
      pair_t[p] = bad_t ? 0 : t;
      pair_wf[p] = w;
      pair_wi[p] = impact == GS_IMPACT_U8 ? quant_u8(w) : 0;
      if (!bad_t && !bad_w && q >= 0 && q < B) {
        const int64_t nb = term_block[t + 1] - term_block[t];
        nch = (nb + chunk_blocks - 1) / chunk_blocks;
      }
    }
    // block exclusive scan of nch (int64)
    int64_t x = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t s = s_wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      s_wsum[lane] = s;
    }
    __syncthreads();
    const int64_t incl = x + (warp > 0 ? s_wsum[warp - 1] : 0) + s_carry;
    if (p < q_nnz) pair_chunk[p] = incl - nch;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = incl;
    __syncthreads();
  }
  (void)warp_buf;
  if (threadIdx.x == 0) {
    pair_chunk[q_nnz] = s_carry;
    hdr->total_chunks = s_carry;
  }
  if (flags) atomicOr(&hdr->flags, flags);
}

__global__ void zero_kernel(uint32_t* __restrict__ p, int64_t words) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = words / 4;
  uint4* p4 = reinterpret_cast<uint4*>(p);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) p4[i] = make_uint4(0, 0, 0, 0);
  for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) p[i] = 0u;
}

// Posting loads are streamed with an L2 evict-first policy, so that the
// score rows the reductions update keep their L2 lines.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ int4 ldg_stream_v4(const void* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint2 ldg_stream_v2(const void* p, uint64_t pol) {
  uint2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ldg_stream_u32(const void* p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

// four impacts of one lane (postings 4j..4j+3 of a block), as float (or int)
template <int IMPACT>
__device__ __forceinline__ void load4_impacts(const uint8_t* blk, int j, float (&x)[4], int (&xi)[4], uint64_t pol) {
  if (IMPACT == GS_IMPACT_F32) {
    int4 v = ldg_stream_v4(blk + 128 + j * 16, pol);
    x[0] = __int_as_float(v.x); x[1] = __int_as_float(v.y); x[2] = __int_as_float(v.z); x[3] = __int_as_float(v.w);
  } else if (IMPACT == GS_IMPACT_F16) {
    uint2 v = ldg_stream_v2(blk + 128 + j * 8, pol);
    __half2 a = *reinterpret_cast<__half2*>(&v.x), b = *reinterpret_cast<__half2*>(&v.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    x[0] = fa.x; x[1] = fa.y; x[2] = fb.x; x[3] = fb.y;
  } else if (IMPACT == GS_IMPACT_BF16) {
    uint2 v = ldg_stream_v2(blk + 128 + j * 8, pol);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&v.x), b = *reinterpret_cast<__nv_bfloat162*>(&v.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    x[0] = fa.x; x[1] = fa.y; x[2] = fb.x; x[3] = fb.y;
  } else {
    uint32_t v = ldg_stream_u32(blk + 128 + j * 4, pol);
    xi[0] = v & 0xff; xi[1] = (v >> 8) & 0xff; xi[2] = (v >> 16) & 0xff; xi[3] = v >> 24;
  }
}

// Each warp walks a work item 4 blocks per step (8 lanes per block, 4
// postings per lane, 128-bit loads).  kUnroll steps are loaded before any of
// their postings is added: 4 steps measured no faster than 1 (the kernel is
// bound by the L2 reduction rate) and halve the resident warps, so 1.
template <int IMPACT>
__global__ void __launch_bounds__(256) tp_scatter_kernel(
    const uint8_t* __restrict__ blocks, const int64_t* __restrict__ term_block, const int32_t* __restrict__ pair_q,
    const int32_t* __restrict__ pair_t, const float* __restrict__ pair_wf, const int32_t* __restrict__ pair_wi,
    const int64_t* __restrict__ pair_chunk, int64_t npairs, const Header* __restrict__ hdr, int chunk_blocks,
    int64_t ld, void* __restrict__ rows) {
  constexpr int bb = block_bytes(IMPACT);
  constexpr int kUnroll = 1;
  const uint64_t pol = evict_first_policy();
  const int lane = threadIdx.x & 31;
  const int j = lane & 7;
  const int64_t total = hdr->total_chunks;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < total; c += nwarps) {
    const int64_t p = upper_bound_i64(pair_chunk, npairs + 1, c) - 1;
    const int q = pair_q[p];
    const int32_t t = pair_t[p];
    const int64_t b_end = term_block[t + 1];
    const int64_t b0 = term_block[t] + (c - pair_chunk[p]) * chunk_blocks;
    const int64_t b1 = min(b0 + chunk_blocks, b_end);
    const float wf = pair_wf[p];
    const int32_t wi = pair_wi[p];
    float* rowf = static_cast<float*>(rows) + (int64_t)q * ld;
    int32_t* rowi = static_cast<int32_t*>(rows) + (int64_t)q * ld;
    for (int64_t b = b0 + (lane >> 3); b < b1; b += 4 * kUnroll) {
      int4 ids[kUnroll];
      float x[kUnroll][4];
      int xi[kUnroll][4];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        ids[u] = make_int4(-1, -1, -1, -1);
        const int64_t bu = b + 4 * u;
        if (bu < b1) {
          const uint8_t* blk = blocks + bu * bb;
          ids[u] = ldg_stream_v4(blk + j * 16, pol);
          load4_impacts<IMPACT>(blk, j, x[u], xi[u], pol);
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int id[4] = {ids[u].x, ids[u].y, ids[u].z, ids[u].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (id[e] < 0) continue;  // padding (and steps past the item)
          if (IMPACT == GS_IMPACT_U8) atomicAdd(rowi + id[e], wi * xi[u][e]);
          else atomicAdd(rowf + id[e], wf * x[u][e]);
        }
      }
    }
  }
}

struct TpPlan {
  Header* hdr;
  int32_t* pair_q;
  int32_t* pair_t;
  float* pair_wf;
  int32_t* pair_wi;
  int64_t* pair_chunk;
  void* rows;  // [B x ld]
  int64_t ld;
  void* topk_ws;  // the dense-row top-k's workspace
  size_t topk_bytes;
};

// Workspace = [term-parallel region (header first)][doc-tiled region][host-io region]
TpPlan carve_tp(void* ws, const gs_index* ix, int32_t B, int64_t q_nnz, bool with_rows, size_t* bytes,
                int32_t k = 1) {
  Carver c(ws);
  TpPlan p{};
  p.hdr = c.take<Header>(1);
  p.pair_q = c.take<int32_t>(q_nnz + 1);
  p.pair_t = c.take<int32_t>(q_nnz + 1);
  p.pair_wf = c.take<float>(q_nnz + 1);
  p.pair_wi = c.take<int32_t>(q_nnz + 1);
  p.pair_chunk = c.take<int64_t>(q_nnz + 1);
  p.ld = (ix->N + 31) / 32 * 32;
  p.rows = with_rows ? (void*)c.take<uint32_t>((size_t)B * p.ld) : nullptr;
  p.topk_bytes = 0;
  if (with_rows) dense_topk_workspace_bytes(ix, B, k, &p.topk_bytes);
  p.topk_ws = p.topk_bytes ? (void*)c.take<uint8_t>(p.topk_bytes) : nullptr;
  *bytes = c.size();
  return p;
}

struct IoPlan {
  int32_t* indptr;
  int32_t* terms;
  float* w;
  int32_t* ids;
  void* scores;
};

IoPlan carve_io(void* base, int32_t B, int64_t q_nnz, int32_t k, size_t* bytes) {
  Carver c(base);
  IoPlan p{};
  p.indptr = c.take<int32_t>(B + 1);
  p.terms = c.take<int32_t>(q_nnz + 1);
  p.w = c.take<float>(q_nnz + 1);
  p.ids = c.take<int32_t>((size_t)B * std::max(k, 1));
  p.scores = c.take<uint32_t>((size_t)B * std::max(k, 1));
  *bytes = c.size();
  return p;
}

int persistent_grid(const gs_index* ix, int per_sm) { return std::max(1, ix->sms) * per_sm; }

template <int IMPACT>
void launch_tp_scatter(const gs_index* ix, const TpPlan& p, int64_t q_nnz, int chunk, void* rows, int64_t ld,
                       cudaStream_t s) {
  tp_scatter_kernel<IMPACT><<<persistent_grid(ix, 8), 256, 0, s>>>(ix->blocks, ix->term_block, p.pair_q, p.pair_t,
                                                                  p.pair_wf, p.pair_wi, p.pair_chunk, q_nnz, p.hdr,
                                                                  chunk, ld, rows);
}

gs_status run_tp_scores(const gs_index* ix, const int32_t* q_indptr, const int32_t* q_terms, const float* q_w,
                        int32_t B, int64_t q_nnz, const TpPlan& p, int chunk, void* rows, int64_t ld,
                        const gs_search_opts* opts, cudaStream_t s) {
  record_stage(opts, 0, s);
  tp_prep_kernel<<<1, kPrepThreads, 0, s>>>(q_indptr, q_terms, q_w, B, q_nnz, ix->V, ix->impact, ix->term_block,
                                            chunk, p.pair_q, p.pair_t, p.pair_wf, p.pair_wi, p.pair_chunk, p.hdr);
  GS_LAUNCH_CHECK();
  record_stage(opts, 1, s);
  const int64_t words = (int64_t)B * ld;
  zero_kernel<<<persistent_grid(ix, 4), 512, 0, s>>>(static_cast<uint32_t*>(rows), words);
  GS_LAUNCH_CHECK();
  record_stage(opts, 2, s);
  record_stage(opts, 3, s);
  switch (ix->impact) {
    case GS_IMPACT_F32: launch_tp_scatter<GS_IMPACT_F32>(ix, p, q_nnz, chunk, rows, ld, s); break;
    case GS_IMPACT_F16: launch_tp_scatter<GS_IMPACT_F16>(ix, p, q_nnz, chunk, rows, ld, s); break;
    case GS_IMPACT_BF16: launch_tp_scatter<GS_IMPACT_BF16>(ix, p, q_nnz, chunk, rows, ld, s); break;
    default: launch_tp_scatter<GS_IMPACT_U8>(ix, p, q_nnz, chunk, rows, ld, s); break;
  }
  GS_LAUNCH_CHECK();
  record_stage(opts, 4, s);
  return GS_OK;
}

gs_status run_topk_dense(const gs_index* ix, const TpPlan& p, int32_t B, int32_t k, int32_t* out_ids,
                         void* out_scores, cudaStream_t s) {
  return dense_topk(ix, p.rows, p.ld, B, k, out_ids, out_scores, p.topk_ws, p.topk_bytes, &p.hdr->flags, s);
}

int resolve_algo(const gs_index* ix, const gs_search_opts* opts) {
  int algo = opts ? opts->algo : GS_ALGO_AUTO;
  if (algo == GS_ALGO_AUTO) algo = ix->seg ? GS_ALGO_DOC_TILED : GS_ALGO_TERM_PARALLEL;
  return algo;
}

gs_status check_query_args(const gs_index* ix, int32_t B, int64_t q_nnz, int32_t k, bool need_k) {
  if (!ix || B < 1 || q_nnz < 0 || q_nnz > INT32_MAX - 1) return GS_ERR_INVALID_ARG;
  if (need_k) {
    if (k < 1 || (int64_t)k > ix->N) return GS_ERR_INVALID_ARG;
    if (k > GS_MAX_K) return GS_ERR_UNSUPPORTED;
  }
  return GS_OK;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_search_workspace_size(const gs_index* ix, int32_t B, int64_t q_nnz, int32_t k,
                                              const gs_search_opts* opts, int32_t host_io, size_t* bytes) {
  if (!bytes) return GS_ERR_INVALID_ARG;
  gs_status st = check_query_args(ix, B, q_nnz, std::max(k, 1), false);
  if (st != GS_OK) return st;
  const int algo = resolve_algo(ix, opts);
  size_t tp_bytes = 0;
  carve_tp(nullptr, ix, B, q_nnz, algo == GS_ALGO_TERM_PARALLEL, &tp_bytes, std::max(k, 1));
  if (algo == GS_ALGO_DOC_PARALLEL) {
    size_t dp = 0;
    st = dp_workspace_bytes(ix, B, &dp);
    if (st != GS_OK) return st;
    tp_bytes += dp;
  }
  if (algo == GS_ALGO_DOC_TILED) {
    size_t dt = 0;
    st = dt_workspace_bytes(ix, B, q_nnz, std::max(k, 1), opts, &dt);
    if (st != GS_OK) return st;
    tp_bytes += dt;
  }
  if (host_io) {
    size_t io = 0;
    carve_io(nullptr, B, q_nnz, std::max(k, 1), &io);
    tp_bytes += io;
  }
  *bytes = tp_bytes;
  return GS_OK;
}

extern "C" gs_status gs_search(const gs_index* ix, const int32_t* q_indptr, const int32_t* q_terms, const float* q_w,
                               int32_t B, int64_t q_nnz, int32_t k, int32_t* out_ids, void* out_scores,
                               void* workspace, size_t workspace_bytes, const gs_search_opts* opts,
                               gs_stream_t stream) {
  gs_status st = check_query_args(ix, B, q_nnz, k, true);
  if (st != GS_OK) return st;
  if (!q_indptr || (q_nnz > 0 && (!q_terms || !q_w)) || !out_ids || !out_scores || !workspace)
    return GS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return GS_ERR_INVALID_ARG;
  size_t need = 0;
  st = gs_search_workspace_size(ix, B, q_nnz, k, opts, 0, &need);
  if (st != GS_OK) return st;
  if (workspace_bytes < need) return GS_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int algo = resolve_algo(ix, opts);
  size_t tp_bytes = 0;
  TpPlan p = carve_tp(workspace, ix, B, q_nnz, algo == GS_ALGO_TERM_PARALLEL, &tp_bytes, k);
  GS_CUDA_TRY(cudaMemsetAsync(p.hdr, 0, sizeof(Header), s));
  if (algo == GS_ALGO_DOC_PARALLEL) {
    return dp_search(ix, q_indptr, q_terms, q_w, B, q_nnz, k, out_ids, out_scores,
                     static_cast<uint8_t*>(workspace) + tp_bytes, workspace_bytes - tp_bytes, &p.hdr->flags, opts, s);
  }
  if (algo == GS_ALGO_DOC_TILED) {
    return dt_search(ix, q_indptr, q_terms, q_w, B, q_nnz, k, out_ids, out_scores,
                     static_cast<uint8_t*>(workspace) + tp_bytes, workspace_bytes - tp_bytes, &p.hdr->flags, opts,
                     s);
  }
  const int chunk = (opts && opts->chunk_blocks > 0) ? opts->chunk_blocks : kDefaultChunkBlocks;
  st = run_tp_scores(ix, q_indptr, q_terms, q_w, B, q_nnz, p, chunk, p.rows, p.ld, opts, s);
  if (st != GS_OK) return st;
  st = run_topk_dense(ix, p, B, k, out_ids, out_scores, s);
  record_stage(opts, 5, s);
  return st;
}

extern "C" gs_status gs_score_dense(const gs_index* ix, const int32_t* q_indptr, const int32_t* q_terms,
                                    const float* q_w, int32_t B, int64_t q_nnz, void* out_rows, void* workspace,
                                    size_t workspace_bytes, gs_stream_t stream) {
  gs_status st = check_query_args(ix, B, q_nnz, 1, false);
  if (st != GS_OK) return st;
  if (!q_indptr || (q_nnz > 0 && (!q_terms || !q_w)) || !out_rows || !workspace) return GS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return GS_ERR_INVALID_ARG;
  gs_search_opts o{};
  o.algo = GS_ALGO_TERM_PARALLEL;
  size_t need = 0;
  st = gs_search_workspace_size(ix, B, q_nnz, 1, &o, 0, &need);
  if (st != GS_OK) return st;
  if (workspace_bytes < need) return GS_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  size_t tp_bytes = 0;
  TpPlan p = carve_tp(workspace, ix, B, q_nnz, false, &tp_bytes);
  GS_CUDA_TRY(cudaMemsetAsync(p.hdr, 0, sizeof(Header), s));
  return run_tp_scores(ix, q_indptr, q_terms, q_w, B, q_nnz, p, kDefaultChunkBlocks, out_rows, ix->N, nullptr, s);
}

extern "C" gs_status gs_search_host(const gs_index* ix, const int32_t* h_q_indptr, const int32_t* h_q_terms,
                                    const float* h_q_w, int32_t B, int64_t q_nnz, int32_t k, int32_t* h_out_ids,
                                    void* h_out_scores, void* workspace, size_t workspace_bytes,
                                    const gs_search_opts* opts, gs_stream_t stream) {
  gs_status st = check_query_args(ix, B, q_nnz, k, true);
  if (st != GS_OK) return st;
  if (!h_q_indptr || (q_nnz > 0 && (!h_q_terms || !h_q_w)) || !h_out_ids || !h_out_scores || !workspace)
    return GS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return GS_ERR_INVALID_ARG;
  size_t need = 0;
  st = gs_search_workspace_size(ix, B, q_nnz, k, opts, 1, &need);
  if (st != GS_OK) return st;
  if (workspace_bytes < need) return GS_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  size_t search_bytes = 0, io_bytes = 0;
  st = gs_search_workspace_size(ix, B, q_nnz, k, opts, 0, &search_bytes);
  if (st != GS_OK) return st;
  // the host-io buffers sit after everything gs_search itself uses
  IoPlan io = carve_io(static_cast<uint8_t*>(workspace) + search_bytes, B, q_nnz, k, &io_bytes);
  GS_CUDA_TRY(cudaMemcpyAsync(io.indptr, h_q_indptr, sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, s));
  if (q_nnz > 0) {
    GS_CUDA_TRY(cudaMemcpyAsync(io.terms, h_q_terms, sizeof(int32_t) * q_nnz, cudaMemcpyHostToDevice, s));
    GS_CUDA_TRY(cudaMemcpyAsync(io.w, h_q_w, sizeof(float) * q_nnz, cudaMemcpyHostToDevice, s));
  }
  st = gs_search(ix, io.indptr, io.terms, io.w, B, q_nnz, k, io.ids, io.scores, workspace, search_bytes, opts,
                 stream);
  if (st != GS_OK) return st;
  GS_CUDA_TRY(cudaMemcpyAsync(h_out_ids, io.ids, sizeof(int32_t) * B * (size_t)k, cudaMemcpyDeviceToHost, s));
  GS_CUDA_TRY(cudaMemcpyAsync(h_out_scores, io.scores, sizeof(uint32_t) * B * (size_t)k, cudaMemcpyDeviceToHost, s));
  uint32_t flags = 0;  // the flag word leads the workspace
  GS_CUDA_TRY(cudaMemcpyAsync(&flags, workspace, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA_TRY(cudaStreamSynchronize(s));
  return flags_status(flags);
}

extern "C" gs_status gs_search_plan(const gs_index* ix, int32_t B, int64_t q_nnz, int32_t k,
                                    const gs_search_opts* opts, gs_plan_info* out) {
  if (!out) return GS_ERR_INVALID_ARG;
  gs_status st = check_query_args(ix, B, q_nnz, k, true);
  if (st != GS_OK) return st;
  std::memset(out, 0, sizeof(*out));
  const int algo = resolve_algo(ix, opts);
  if (algo == GS_ALGO_DOC_TILED) return dt_plan_info(ix, B, k, opts, out);
  if (algo == GS_ALGO_DOC_PARALLEL && !ix->dm_indptr) return GS_ERR_UNSUPPORTED;
  out->algo = algo;
  out->chunk_blocks = (opts && opts->chunk_blocks > 0) ? opts->chunk_blocks : kDefaultChunkBlocks;
  return GS_OK;
}

extern "C" gs_status gs_search_query_order(const gs_index* ix, int32_t B, int64_t q_nnz, int32_t k,
                                           const gs_search_opts* opts, const void* workspace, size_t workspace_bytes,
                                           int32_t* out_perm, gs_stream_t stream) {
  gs_status st = check_query_args(ix, B, q_nnz, k, true);
  if (st != GS_OK) return st;
  if (!workspace || !out_perm) return GS_ERR_INVALID_ARG;
  if (resolve_algo(ix, opts) != GS_ALGO_DOC_TILED) return GS_ERR_UNSUPPORTED;
  size_t tp_bytes = 0;
  carve_tp(nullptr, ix, B, q_nnz, false, &tp_bytes, k);
  if (workspace_bytes < tp_bytes) return GS_ERR_WORKSPACE;
  return dt_order_of(ix, B, q_nnz, k, opts, static_cast<const uint8_t*>(workspace) + tp_bytes,
                     workspace_bytes - tp_bytes, out_perm, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" gs_status gs_search_flags(const void* workspace, gs_stream_t stream, uint32_t* flags) {
  if (!workspace || !flags) return GS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  GS_CUDA_TRY(cudaStreamSynchronize(s));
  GS_CUDA_TRY(cudaMemcpy(flags, workspace, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  return GS_OK;
}
