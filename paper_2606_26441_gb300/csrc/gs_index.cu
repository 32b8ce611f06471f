// Index build (Sec. 3.2): term-major, doc-sorted posting lists padded to W = 32,
// stored as 32-posting blocks [32 x int32 doc id][32 x impact], plus per-term
// metadata (Eq. 2 padded lengths, max impacts) and the per-tile segment table
// the doc-tiled kernel uses.
//
// Steps (all on the caller's stream):
//   1. validate the document CSR;
//   2. split the documents into C chunks and count, per (chunk, term), the
//      postings of the chunk (global atomics);
//   3. turn the counts into per-(chunk, term) base positions inside each
//      term's list (prefix over chunks) -> list lengths;
//   4. prefix over terms of the block counts -> block offset of each list;
//   5. each warp walks its chunk's documents in increasing id and appends
//      their postings at the running positions: lists come out doc-sorted;
//   6. per term: order/duplicate check, max impact, segment table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "gs_doctiled.cuh"
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr uint32_t kErrIndptr = 1, kErrTerm = 2, kErrWeight = 4, kErrDup = 8;

__global__ void validate_docs_kernel(const int64_t* __restrict__ indptr, const int32_t* __restrict__ terms,
                                     const float* __restrict__ w, int64_t N, int64_t nnz, int32_t V,
                                     int impact, uint32_t* err) {
  uint32_t e = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t d = tid; d < N; d += stride) {
    int64_t a = indptr[d], b = indptr[d + 1];
    if (b < a || a < 0 || b > nnz) e |= kErrIndptr;
    if (d == 0 && a != 0) e |= kErrIndptr;
    if (d == N - 1 && b != nnz) e |= kErrIndptr;
  }
  for (int64_t p = tid; p < nnz; p += stride) {
    int32_t t = terms[p];
    float x = w[p];
    if (t < 0 || t >= V) e |= kErrTerm;
    if (!isfinite(x)) e |= kErrWeight;
    if (impact == GS_IMPACT_U8 && !(x >= 0.0f && x <= 5.0f)) e |= kErrWeight;
    if (impact == GS_IMPACT_F16 && isinf(__half2float(__float2half_rn(x)))) e |= kErrWeight;
  }
  if (e) atomicOr(err, e);
}

// cnt[c * V + t] += 1 for every posting of every document of chunk c
__global__ void count_kernel(const int64_t* __restrict__ indptr, const int32_t* __restrict__ terms,
                             int64_t N, int32_t V, int64_t docs_per_chunk, uint32_t* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += stride) {
    uint32_t* row = cnt + (d / docs_per_chunk) * (int64_t)V;
    for (int64_t p = indptr[d]; p < indptr[d + 1]; ++p) atomicAdd(&row[terms[p]], 1u);
  }
}

// per term: cnt[c][t] <- postings of t in chunks < c; len[t] = total
__global__ void chunk_prefix_kernel(uint32_t* __restrict__ cnt, int64_t C, int32_t V,
                                    int32_t* __restrict__ term_len, int64_t* __restrict__ nblk) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= V) return;
  uint32_t run = 0;
  for (int64_t c = 0; c < C; ++c) {
    uint32_t v = cnt[c * V + t];
    cnt[c * V + t] = run;
    run += v;
  }
  term_len[t] = (int32_t)run;
  nblk[t] = ((int64_t)run + kBlock - 1) / kBlock;
}

// exclusive prefix of nblk[0..V) into out[0..V]; one CTA of 1024 threads
__global__ void block_offsets_kernel(const int64_t* __restrict__ nblk, int32_t V, int64_t* __restrict__ out) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < V; base += blockDim.x) {
    int i = base + threadIdx.x;
    int64_t v = (i < V) ? nblk[i] : 0;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t s = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    int64_t incl = x + (warp > 0 ? warp_sums[warp - 1] : 0) + carry;
    if (i < V) out[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[V] = carry;
}

// every id slot -1, every impact 0 (padding, Sec. 3.2); postings overwrite
__global__ void init_blocks_kernel(uint8_t* __restrict__ blocks, int64_t nblocks, int impact) {
  const int bb = block_bytes(impact);
  const int64_t words = nblocks * (int64_t)bb / 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t* w = reinterpret_cast<uint32_t*>(blocks);
  const int words_per_block = bb / 4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) {
    int in_block = (int)(i % words_per_block);
    w[i] = in_block < 32 ? 0xFFFFFFFFu : 0u;
  }
}

template <int IMPACT>
__device__ __forceinline__ void store_impact(uint8_t* blk, int lane_in, float x) {
  if (IMPACT == GS_IMPACT_F32) {
    reinterpret_cast<float*>(blk + 128)[lane_in] = x;
  } else if (IMPACT == GS_IMPACT_F16) {
    reinterpret_cast<__half*>(blk + 128)[lane_in] = __float2half_rn(x);
  } else if (IMPACT == GS_IMPACT_BF16) {
    reinterpret_cast<__nv_bfloat16*>(blk + 128)[lane_in] = __float2bfloat16_rn(x);
  } else {
    (blk + 128)[lane_in] = (uint8_t)quant_u8(x);
  }
}

// one warp per chunk: documents in increasing id, postings at running positions
template <int IMPACT>
__global__ void scatter_kernel(const int64_t* __restrict__ indptr, const int32_t* __restrict__ terms,
                               const float* __restrict__ w, int64_t N, int32_t V, int64_t docs_per_chunk,
                               int64_t C, uint32_t* __restrict__ cnt, const int64_t* __restrict__ term_block,
                               uint8_t* __restrict__ blocks) {
  const int lane = threadIdx.x & 31;
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= C) return;
  constexpr int bb = block_bytes(IMPACT);
  uint32_t* run = cnt + c * (int64_t)V;
  const int64_t d0 = c * docs_per_chunk;
  const int64_t d1 = min(N, d0 + docs_per_chunk);
  for (int64_t d = d0; d < d1; ++d) {
    const int64_t a = indptr[d], b = indptr[d + 1];
    for (int64_t p = a + lane; p < b; p += 32) {
      const int32_t t = terms[p];
      const uint32_t pos = run[t];
      run[t] = pos + 1;
      uint8_t* blk = blocks + (term_block[t] + pos / kBlock) * bb;
      const int li = (int)(pos % kBlock);
      reinterpret_cast<int32_t*>(blk)[li] = (int32_t)d;
      store_impact<IMPACT>(blk, li, w[p]);
    }
    __syncwarp();
  }
}

template <int IMPACT>
__device__ __forceinline__ float load_impact(const uint8_t* blk, int li) {
  if (IMPACT == GS_IMPACT_F32) return reinterpret_cast<const float*>(blk + 128)[li];
  if (IMPACT == GS_IMPACT_F16) return __half2float(reinterpret_cast<const __half*>(blk + 128)[li]);
  if (IMPACT == GS_IMPACT_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(blk + 128)[li]);
  return (float)(blk + 128)[li];
}

// one CTA per term: doc order / duplicates, max impact, segment table
template <int IMPACT>
__global__ void finalize_kernel(const uint8_t* __restrict__ blocks, const int64_t* __restrict__ term_block,
                                const int32_t* __restrict__ term_len, int32_t V, int tile_docs,
                                int num_tiles, float* __restrict__ max_score, float* __restrict__ max_abs,
                                uint32_t* __restrict__ seg, uint32_t* err) {
  const int t = blockIdx.x;
  constexpr int bb = block_bytes(IMPACT);
  const int64_t len = term_len[t];
  const uint8_t* base = blocks + term_block[t] * bb;
  uint32_t* srow = seg ? seg + (int64_t)t * (num_tiles + 1) : nullptr;
  float mx = -INFINITY, ma = 0.0f;
  uint32_t e = 0;
  for (int64_t p = threadIdx.x; p < len; p += blockDim.x) {
    const uint8_t* blk = base + (p / kBlock) * bb;
    const int32_t doc = reinterpret_cast<const int32_t*>(blk)[p % kBlock];
    const float xv = load_impact<IMPACT>(blk, (int)(p % kBlock));
    mx = fmaxf(mx, xv);
    ma = fmaxf(ma, fabsf(xv));
    int32_t prev = -1;
    if (p > 0) {
      const uint8_t* pb = base + ((p - 1) / kBlock) * bb;
      prev = reinterpret_cast<const int32_t*>(pb)[(p - 1) % kBlock];
    }
    if (doc < 0 || doc <= prev) e |= kErrDup;
    if (srow && doc >= 0) {
      const int tile = doc / tile_docs;
      const int prev_tile = (p > 0 && prev >= 0) ? prev / tile_docs : -1;
      for (int j = prev_tile + 1; j <= tile && j <= num_tiles; ++j) srow[j] = (uint32_t)p;
      if (p == len - 1)
        for (int j = tile + 1; j <= num_tiles; ++j) srow[j] = (uint32_t)len;
    }
  }
  if (len == 0 && srow)
    for (int j = threadIdx.x; j <= num_tiles; j += blockDim.x) srow[j] = 0u;
  // block maxima
  __shared__ float red[32], red_a[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = mx;
    red_a[threadIdx.x >> 5] = ma;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = -INFINITY, a = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      m = fmaxf(m, red[i]);
      a = fmaxf(a, red_a[i]);
    }
    max_score[t] = len > 0 ? m : 0.0f;
    max_abs[t] = a;
  }
  if (e) atomicOr(err, e);
}

// Dense head: row h holds, for every document, the stored impact of term
// head_term[h] (0 where the document lacks it).  One CTA per head term.
__global__ void head_fill_kernel(const uint8_t* __restrict__ blocks, const int64_t* __restrict__ term_block,
                                 const int32_t* __restrict__ term_len, const int32_t* __restrict__ head_term,
                                 int impact, int64_t head_ld, uint8_t* __restrict__ head_dense) {
  const int h = blockIdx.x;
  const int32_t t = head_term[h];
  const int ib = impact_bytes(impact);
  const int bb = block_bytes(impact);
  const uint8_t* base = blocks + term_block[t] * bb;
  uint8_t* row = head_dense + (int64_t)h * head_ld * ib;
  for (int64_t p = threadIdx.x; p < term_len[t]; p += blockDim.x) {
    const uint8_t* blk = base + (p / kBlock) * bb;
    const int li = (int)(p % kBlock);
    const int32_t doc = reinterpret_cast<const int32_t*>(blk)[li];
    if (doc < 0 || doc >= head_ld) continue;  // only valid lists reach here; stay in bounds regardless
    for (int b = 0; b < ib; ++b) row[(int64_t)doc * ib + b] = blk[128 + li * ib + b];
  }
}

// document-major copy: the caller's doc CSR with stored (converted) impacts
template <int IMPACT>
__global__ void doc_major_kernel(const float* __restrict__ w, int64_t nnz, uint8_t* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const float x = w[p];
    if (IMPACT == GS_IMPACT_F32) reinterpret_cast<float*>(out)[p] = x;
    else if (IMPACT == GS_IMPACT_F16) reinterpret_cast<__half*>(out)[p] = __float2half_rn(x);
    else if (IMPACT == GS_IMPACT_BF16) reinterpret_cast<__nv_bfloat16*>(out)[p] = __float2bfloat16_rn(x);
    else out[p] = (uint8_t)quant_u8(x);
  }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

int grid_for(int64_t n, int threads, int sms) {
  int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms * 16));
}

template <int IMPACT>
void launch_scatter(const int64_t* indptr, const int32_t* terms, const float* w, int64_t N, int32_t V,
                    int64_t dpc, int64_t C, uint32_t* cnt, const int64_t* term_block, uint8_t* blocks,
                    cudaStream_t s) {
  int threads = 128;
  int grid = (int)((C * 32 + threads - 1) / threads);
  scatter_kernel<IMPACT><<<grid, threads, 0, s>>>(indptr, terms, w, N, V, dpc, C, cnt, term_block, blocks);
}

template <int IMPACT>
void launch_finalize(const uint8_t* blocks, const int64_t* term_block, const int32_t* term_len, int32_t V,
                     int tile_docs, int num_tiles, float* max_score, float* max_abs, uint32_t* seg,
                     uint32_t* err, cudaStream_t s) {
  finalize_kernel<IMPACT><<<V, 256, 0, s>>>(blocks, term_block, term_len, V, tile_docs, num_tiles,
                                            max_score, max_abs, seg, err);
}

}  // namespace
}  // namespace gs

using namespace gs;

static void free_index(gs_index* ix) {
  if (!ix) return;
  cudaFree(ix->blocks);
  cudaFree(ix->term_block);
  cudaFree(ix->term_len);
  cudaFree(ix->max_score);
  cudaFree(ix->max_abs);
  cudaFree(ix->seg);
  cudaFree(ix->head_term);
  cudaFree(ix->head_slot);
  cudaFree(ix->head_dense);
  cudaFree(ix->dm_indptr);
  cudaFree(ix->dm_terms);
  cudaFree(ix->dm_impacts);
  delete ix;
}

extern "C" gs_status gs_index_build_ex(const int64_t* doc_indptr, const int32_t* doc_terms, const float* doc_w,
                                       int64_t num_docs, int64_t nnz, int32_t vocab, gs_impact impact,
                                       const gs_build_opts* opts, gs_stream_t stream, gs_index** out) {
  if (!out) return GS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!doc_indptr || num_docs < 1 || num_docs > INT32_MAX - 1 || nnz < 0 || vocab < 1 ||
      impact < GS_IMPACT_F32 || impact > GS_IMPACT_U8)
    return GS_ERR_INVALID_ARG;
  if (nnz > 0 && (!doc_terms || !doc_w)) return GS_ERR_INVALID_ARG;
  int tile_docs = 1024;
  if (opts && opts->tile_docs != 0) tile_docs = opts->tile_docs;
  if (tile_docs != -1 && (tile_docs < 256 || tile_docs > 65536 || (tile_docs & (tile_docs - 1))))
    return GS_ERR_INVALID_ARG;
  // default head: 24 terms when the head runs on CUDA-core FMAs (FP32 impacts),
  // 64 when it runs on the tensor cores (FP16, BF16, uint8), where rows are cheap
  // (the sizes measured fastest at 8.84M documents)
  int head_req = impact == GS_IMPACT_F32 ? 24 : 64;
  if (opts && opts->head_terms != 0) head_req = opts->head_terms;
  if (head_req < -1 || head_req > GS_MAX_HEAD_TERMS) return GS_ERR_INVALID_ARG;
  if (head_req < 0 || tile_docs < 0) head_req = 0;  // the head serves the doc-tiled kernel only
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  gs_index* ix = new gs_index();
  ix->N = num_docs;
  ix->V = vocab;
  ix->impact = impact;
  ix->nnz = nnz;
  ix->blk_bytes = block_bytes(impact);
  GS_CUDA_TRY(cudaGetDevice(&ix->device));
  ix->sms = device_sm_count(ix->device);
  const int sms = ix->sms;

  auto fail = [&](gs_status st) {
    free_index(ix);
    return st;
  };
  auto cuda_fail = [&](cudaError_t e) {
    set_cuda_error(e);
    free_index(ix);
    return e == cudaErrorMemoryAllocation ? GS_ERR_OUT_OF_MEMORY : GS_ERR_CUDA;
  };

  DevBuf errb, cntb, nblkb;
  cudaError_t e;
  if ((e = cudaMalloc(&errb.p, sizeof(uint32_t))) != cudaSuccess) return cuda_fail(e);
  uint32_t* err = static_cast<uint32_t*>(errb.p);
  if ((e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s)) != cudaSuccess) return cuda_fail(e);

  // 1. validate
  validate_docs_kernel<<<grid_for(std::max(num_docs, nnz), 256, sms), 256, 0, s>>>(
      doc_indptr, doc_terms, doc_w, num_docs, nnz, vocab, impact, err);
  uint32_t herr = 0;
  if ((e = cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
  if (herr) return fail(GS_ERR_DATA);

  // 2. chunk counts (count matrix capped near 256 MB)
  int64_t C = std::max<int64_t>(1, std::min<int64_t>((num_docs + 63) / 64, std::max<int64_t>(1, (64ll << 20) / vocab)));
  const int64_t dpc = (num_docs + C - 1) / C;
  C = (num_docs + dpc - 1) / dpc;
  if ((e = cudaMalloc(&cntb.p, sizeof(uint32_t) * C * vocab)) != cudaSuccess) return cuda_fail(e);
  uint32_t* cnt = static_cast<uint32_t*>(cntb.p);
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * C * vocab, s)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMalloc(&ix->term_len, sizeof(int32_t) * vocab)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMalloc(&nblkb.p, sizeof(int64_t) * vocab)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMalloc(&ix->term_block, sizeof(int64_t) * (vocab + 1))) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMalloc(&ix->max_score, sizeof(float) * vocab)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMalloc(&ix->max_abs, sizeof(float) * vocab)) != cudaSuccess) return cuda_fail(e);
  if (nnz > 0)
    count_kernel<<<grid_for(num_docs, 256, sms), 256, 0, s>>>(doc_indptr, doc_terms, num_docs, vocab, dpc, cnt);
  // 3. per-(chunk, term) bases, list lengths
  chunk_prefix_kernel<<<(vocab + 255) / 256, 256, 0, s>>>(cnt, C, vocab, ix->term_len,
                                                          static_cast<int64_t*>(nblkb.p));
  // 4. block offsets of the lists
  block_offsets_kernel<<<1, 1024, 0, s>>>(static_cast<int64_t*>(nblkb.p), vocab, ix->term_block);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  ix->h_term_block.resize(vocab + 1);
  ix->h_term_len.resize(vocab);
  if ((e = cudaMemcpyAsync(ix->h_term_block.data(), ix->term_block, sizeof(int64_t) * (vocab + 1),
                           cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaMemcpyAsync(ix->h_term_len.data(), ix->term_len, sizeof(int32_t) * vocab, cudaMemcpyDeviceToHost,
                           s)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
  ix->total_blocks = ix->h_term_block[vocab];
  // block indices are kept as int32 by the scoring kernels (2^31 blocks would be
  // 68.7 G postings, more than the device holds)
  if (ix->total_blocks > (int64_t)INT32_MAX) return fail(GS_ERR_UNSUPPORTED);

  // 5. blocks: padding everywhere, then postings in doc order
  const int64_t nb_alloc = std::max<int64_t>(ix->total_blocks, 1);
  if ((e = cudaMalloc(&ix->blocks, nb_alloc * ix->blk_bytes)) != cudaSuccess) return cuda_fail(e);
  init_blocks_kernel<<<grid_for(nb_alloc * ix->blk_bytes / 4, 256, sms), 256, 0, s>>>(ix->blocks, nb_alloc, impact);
  if (nnz > 0) {
    switch (impact) {
      case GS_IMPACT_F32:
        launch_scatter<GS_IMPACT_F32>(doc_indptr, doc_terms, doc_w, num_docs, vocab, dpc, C, cnt, ix->term_block,
                                      ix->blocks, s);
        break;
      case GS_IMPACT_F16:
        launch_scatter<GS_IMPACT_F16>(doc_indptr, doc_terms, doc_w, num_docs, vocab, dpc, C, cnt, ix->term_block,
                                      ix->blocks, s);
        break;
      case GS_IMPACT_BF16:
        launch_scatter<GS_IMPACT_BF16>(doc_indptr, doc_terms, doc_w, num_docs, vocab, dpc, C, cnt,
                                       ix->term_block, ix->blocks, s);
        break;
      default:
        launch_scatter<GS_IMPACT_U8>(doc_indptr, doc_terms, doc_w, num_docs, vocab, dpc, C, cnt, ix->term_block,
                                     ix->blocks, s);
        break;
    }
  }
  // 6. per-term finalisation and the segment table
  if (tile_docs > 0) {
    ix->tile_docs = tile_docs;
    ix->num_tiles = (int32_t)((num_docs + tile_docs - 1) / tile_docs);
    const size_t seg_bytes = sizeof(uint32_t) * (size_t)vocab * (ix->num_tiles + 1);
    if ((e = cudaMalloc(&ix->seg, seg_bytes)) != cudaSuccess) return cuda_fail(e);
    ix->meta_bytes += (int64_t)seg_bytes;
  }
  ix->meta_bytes += (int64_t)vocab * (8 + 4 + 4 + 4) + 8;
  switch (impact) {
    case GS_IMPACT_F32:
      launch_finalize<GS_IMPACT_F32>(ix->blocks, ix->term_block, ix->term_len, vocab, ix->tile_docs, ix->num_tiles,
                                     ix->max_score, ix->max_abs, ix->seg, err, s);
      break;
    case GS_IMPACT_F16:
      launch_finalize<GS_IMPACT_F16>(ix->blocks, ix->term_block, ix->term_len, vocab, ix->tile_docs, ix->num_tiles,
                                     ix->max_score, ix->max_abs, ix->seg, err, s);
      break;
    case GS_IMPACT_BF16:
      launch_finalize<GS_IMPACT_BF16>(ix->blocks, ix->term_block, ix->term_len, vocab, ix->tile_docs,
                                      ix->num_tiles, ix->max_score, ix->max_abs, ix->seg, err, s);
      break;
    default:
      launch_finalize<GS_IMPACT_U8>(ix->blocks, ix->term_block, ix->term_len, vocab, ix->tile_docs, ix->num_tiles,
                                    ix->max_score, ix->max_abs, ix->seg, err, s);
      break;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
  if (herr) return fail(GS_ERR_DATA);
  // dense head: the head_req longest lists (ties: lower term id)
  if (head_req > 0) {
    std::vector<int32_t> order(vocab);
    for (int32_t t = 0; t < vocab; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return ix->h_term_len[a] > ix->h_term_len[b]; });
    int H = 0;
    while (H < head_req && H < vocab && ix->h_term_len[order[H]] > 0) ++H;
    if (H > 0) {
      ix->head_H = H;
      ix->head_ld = (num_docs + 65535) / 65536 * 65536;  // every tile of every size reads in bounds
      std::vector<int32_t> slot(vocab, -1);
      for (int h = 0; h < H; ++h) slot[order[h]] = h;
      const size_t hbytes = (size_t)H * ix->head_ld * impact_bytes(impact);
      if ((e = cudaMalloc(&ix->head_term, sizeof(int32_t) * H)) != cudaSuccess) return cuda_fail(e);
      if ((e = cudaMalloc(&ix->head_slot, sizeof(int32_t) * vocab)) != cudaSuccess) return cuda_fail(e);
      if ((e = cudaMalloc(&ix->head_dense, hbytes)) != cudaSuccess) return cuda_fail(e);
      if ((e = cudaMemcpyAsync(ix->head_term, order.data(), sizeof(int32_t) * H, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
        return cuda_fail(e);
      if ((e = cudaMemcpyAsync(ix->head_slot, slot.data(), sizeof(int32_t) * vocab, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
        return cuda_fail(e);
      if ((e = cudaMemsetAsync(ix->head_dense, 0, hbytes, s)) != cudaSuccess) return cuda_fail(e);
      head_fill_kernel<<<H, 512, 0, s>>>(ix->blocks, ix->term_block, ix->term_len, ix->head_term, impact,
                                         ix->head_ld, ix->head_dense);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
      ix->meta_bytes += (int64_t)(sizeof(int32_t) * (H + vocab));
      // the host copies must outlive the asynchronous uploads
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
    }
  }
  if (opts && opts->doc_major) {
    const int ib = impact_bytes(impact);
    if ((e = cudaMalloc(&ix->dm_indptr, sizeof(int64_t) * (num_docs + 1))) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMalloc(&ix->dm_terms, sizeof(int32_t) * std::max<int64_t>(nnz, 1))) != cudaSuccess)
      return cuda_fail(e);
    if ((e = cudaMalloc(&ix->dm_impacts, (size_t)ib * std::max<int64_t>(nnz, 1))) != cudaSuccess)
      return cuda_fail(e);
    if ((e = cudaMemcpyAsync(ix->dm_indptr, doc_indptr, sizeof(int64_t) * (num_docs + 1), cudaMemcpyDeviceToDevice,
                             s)) != cudaSuccess)
      return cuda_fail(e);
    if (nnz > 0) {
      if ((e = cudaMemcpyAsync(ix->dm_terms, doc_terms, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s)) !=
          cudaSuccess)
        return cuda_fail(e);
      const int grid = grid_for(nnz, 256, sms);
      switch (impact) {
        case GS_IMPACT_F32: doc_major_kernel<GS_IMPACT_F32><<<grid, 256, 0, s>>>(doc_w, nnz, ix->dm_impacts); break;
        case GS_IMPACT_F16: doc_major_kernel<GS_IMPACT_F16><<<grid, 256, 0, s>>>(doc_w, nnz, ix->dm_impacts); break;
        case GS_IMPACT_BF16: doc_major_kernel<GS_IMPACT_BF16><<<grid, 256, 0, s>>>(doc_w, nnz, ix->dm_impacts); break;
        default: doc_major_kernel<GS_IMPACT_U8><<<grid, 256, 0, s>>>(doc_w, nnz, ix->dm_impacts); break;
      }
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    ix->meta_bytes += (int64_t)(num_docs + 1) * 8 + nnz * (4 + ib);
  }
  if ((e = cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
  if (herr) return fail(GS_ERR_DATA);
  // the doc-tiled kernels' shared-memory ceilings are raised here, once per
  // device and form, so that no search (which a caller may capture into a
  // graph) makes the attribute calls
  if (ix->seg) {
    const gs_status st = dt_prepare_device(ix);
    if (st != GS_OK) return fail(st);
  }
  *out = ix;
  return GS_OK;
}

extern "C" gs_status gs_index_build(const int64_t* doc_indptr, const int32_t* doc_terms, const float* doc_w,
                                    int64_t num_docs, int64_t nnz, int32_t vocab, gs_impact impact,
                                    gs_stream_t stream, gs_index** out) {
  return gs_index_build_ex(doc_indptr, doc_terms, doc_w, num_docs, nnz, vocab, impact, nullptr, stream, out);
}

extern "C" gs_status gs_index_info(const gs_index* ix, gs_index_stats* out) {
  if (!ix || !out) return GS_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->num_docs = ix->N;
  out->postings = ix->nnz;
  out->blocks = ix->total_blocks;
  out->padded_postings = ix->total_blocks * kBlock;
  out->posting_bytes = ix->total_blocks * ix->blk_bytes;
  out->meta_bytes = ix->meta_bytes;
  out->vocab = ix->V;
  out->impact = ix->impact;
  out->block_bytes = ix->blk_bytes;
  out->tile_docs = ix->tile_docs;
  out->num_tiles = ix->num_tiles;
  out->score_is_int = ix->impact == GS_IMPACT_U8 ? 1 : 0;
  out->head_terms = ix->head_H;
  out->head_bytes = (int64_t)ix->head_H * ix->head_ld * impact_bytes(ix->impact);
  return GS_OK;
}

extern "C" gs_status gs_index_get_layout(const gs_index* ix, gs_index_layout* out) {
  if (!ix || !out) return GS_ERR_INVALID_ARG;
  out->blocks = ix->blocks;
  out->term_block = ix->term_block;
  out->term_len = ix->term_len;
  out->max_score = ix->max_score;
  out->seg = ix->seg;
  out->head_term = ix->head_term;
  out->head_dense = ix->head_dense;
  out->head_ld = ix->head_ld;
  out->doc_indptr = ix->dm_indptr;
  out->doc_terms = ix->dm_terms;
  out->doc_impacts = ix->dm_impacts;
  return GS_OK;
}

extern "C" void gs_index_free(gs_index* ix) { free_index(ix); }
