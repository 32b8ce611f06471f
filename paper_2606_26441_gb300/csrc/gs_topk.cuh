// Exact top-k of dense score rows (one CTA per row): radix select of the k-th
// largest 32-bit key (11 + 11 + 10 bit digits), an in-order collection pass
// that keeps every key above the threshold and the lowest-id keys equal to it,
// and a bitonic sort of the k winners by (key desc, id asc).
#pragma once

#include <type_traits>

#include "gs_internal.cuh"

namespace gs {

constexpr int kTopkThreads = 1024;
constexpr int kHistCopies = 4;

template <typename ST>
__device__ __forceinline__ ST key_to_score(uint32_t k);
template <>
__device__ __forceinline__ float key_to_score<float>(uint32_t k) {
  return key_to_float(k);
}
template <>
__device__ __forceinline__ int32_t key_to_score<int32_t>(uint32_t k) {
  return key_to_int(k);
}

// block-wide exclusive scan of one int per thread (1024 threads); returns the
// exclusive prefix and writes the block total to *total
__device__ __forceinline__ int block_excl_scan(int v, int* warp_buf, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_buf[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = (lane < (int)(blockDim.x >> 5)) ? warp_buf[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_buf[lane] = s;
  }
  __syncthreads();
  int excl = x - v + (warp > 0 ? warp_buf[warp - 1] : 0);
  *total = warp_buf[(blockDim.x >> 5) - 1];
  __syncthreads();
  return excl;
}

// Sort n_pad (power of two, <= GS_MAX_K) (key, id) pairs in shared memory by
// key descending, id ascending.
__device__ __forceinline__ void bitonic_sort_desc(uint32_t* key, int32_t* id, int n_pad) {
  for (int size = 2; size <= n_pad; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int i = threadIdx.x; i < (n_pad >> 1); i += blockDim.x) {
        int lo = 2 * i - (i & (stride - 1));
        int hi = lo + stride;
        const bool fwd = ((lo & size) == 0);  // this run ends up in final order
        uint32_t ka = key[lo], kb = key[hi];
        int32_t ia = id[lo], ib = id[hi];
        // does a precede b in the final order (key desc, id asc)?
        const bool a_first = (ka > kb) || (ka == kb && (uint32_t)ia < (uint32_t)ib);
        const bool swap = fwd ? !a_first : a_first;
        if (swap) {
          key[lo] = kb; key[hi] = ka;
          id[lo] = ib; id[hi] = ia;
        }
      }
    }
  }
  __syncthreads();
}

// The k largest of n candidates by (key desc, id asc), found by a radix
// select on the composite 64-bit key (key << 32) | ~id, which is distinct for
// distinct ids.  get(i) returns candidate i as (key, id).  Leaves the k
// winners, unordered, in ck / cid (shared memory) and returns after a
// block-wide barrier.  Needs blockDim.x = 1024 and n >= k.
template <class Get>
__device__ __forceinline__ void select_topk_candidates(Get get, int64_t n, int k, uint32_t* hist, int* warp_buf,
                                                       uint32_t* s_digit, int* s_need, int* s_fill, uint32_t* ck,
                                                       int32_t* cid) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) *s_fill = 0;
  __syncthreads();
  uint64_t prefix = 0, pmask = 0;
  int need = k;
  int shift = 64;
  bool done = false;
  const int64_t iters = (n + blockDim.x - 1) / blockDim.x;
  while (!done && shift > 0) {
    const int bits = shift >= 11 ? 11 : shift;
    shift -= bits;
    const int nb = 1 << bits;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int64_t itn = 0; itn < iters; ++itn) {
      const int64_t i = itn * blockDim.x + threadIdx.x;
      int bin = -1;
      if (i < n) {
        const uint2 v = get(i);
        const uint64_t K = ((uint64_t)v.x << 32) | (uint64_t)(~v.y);
        if ((K & pmask) == prefix) bin = (int)((K >> shift) & (uint64_t)(nb - 1));
      }
      const unsigned peers = __match_any_sync(0xffffffffu, bin);
      if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
    }
    __syncthreads();
    const int per = (nb + (int)blockDim.x - 1) / (int)blockDim.x;
    int local = 0;
    for (int u = 0; u < per; ++u) {
      const int b = nb - 1 - ((int)threadIdx.x * per + u);
      if (b >= 0) local += (int)hist[b];
    }
    int tot;
    int acc = block_excl_scan(local, warp_buf, &tot);
    for (int u = 0; u < per; ++u) {
      const int b = nb - 1 - ((int)threadIdx.x * per + u);
      if (b < 0) break;
      const int h = (int)hist[b];
      if (acc < need && need <= acc + h) {
        *s_digit = (uint32_t)b;
        *s_need = need - acc;
      }
      acc += h;
    }
    __syncthreads();
    const uint32_t D = *s_digit;
    const int new_need = *s_need;
    __syncthreads();
    prefix |= (uint64_t)D << shift;
    pmask |= (uint64_t)(nb - 1) << shift;
    if (new_need == (int)hist[D]) done = true;  // every key in bin D is taken
    need = new_need;
    __syncthreads();
  }
  // every candidate whose composite key, cut to the resolved bits, is >= prefix
  for (int64_t itn = 0; itn < iters; ++itn) {
    const int64_t i = itn * blockDim.x + threadIdx.x;
    if (i < n) {
      const uint2 v = get(i);
      const uint64_t K = ((uint64_t)v.x << 32) | (uint64_t)(~v.y);
      if ((K & pmask) >= prefix) {
        const int slot = atomicAdd(s_fill, 1);
        if (slot < k) {
          ck[slot] = v.x;
          cid[slot] = (int32_t)v.y;
        }
      }
    }
  }
  __syncthreads();
}

// The k-th largest 32-bit key of row r[0..N) (radix select, 11 + 11 + 10 bit
// digits, one histogram pass over the row per digit).  *need_out receives how
// many keys equal to it belong to the top k.  blockDim.x must be 1024.
template <typename ST>
__device__ __forceinline__ uint32_t radix_kth_key(const ST* __restrict__ r, int64_t N, int k,
                                                  uint32_t (*hist)[2048], int* warp_buf, uint32_t* s_digit_p,
                                                  int* s_need_p, int* need_out, int passes = 3) {
  uint32_t& s_digit = *s_digit_p;
  int& s_need = *s_need_p;
  const int lane = threadIdx.x & 31;
  const int copy = (threadIdx.x >> 5) % kHistCopies;
  uint32_t prefix = 0, pmask = 0;
  int need = k;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
    const int nb = pass == 2 ? 1024 : 2048;
    for (int i = threadIdx.x; i < kHistCopies * 2048; i += blockDim.x) (&hist[0][0])[i] = 0;
    __syncthreads();
    // uniform trip count across the block so that every lane reaches the match
    const int64_t iters = (N + blockDim.x - 1) / blockDim.x;
    for (int64_t it = 0; it < iters; ++it) {
      const int64_t i = it * blockDim.x + threadIdx.x;
      int bin = -1;
      if (i < N) {
        const uint32_t key = score_key(r[i]);
        if ((key & pmask) == prefix) bin = (int)((key >> shift) & (uint32_t)(nb - 1));
      }
      const unsigned peers = __match_any_sync(0xffffffffu, bin);
      if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[copy][bin], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      uint32_t s = 0;
#pragma unroll
      for (int c = 0; c < kHistCopies; ++c) s += hist[c][b];
      hist[0][b] = s;
    }
    __syncthreads();
    // digit D: number of matching keys with digit > D is < need <= that + hist[D].
    // Thread j owns bins [2j, 2j + 1] counted from the top (bin nb-1-2j, nb-2-2j).
    {
      const int per = nb / (int)blockDim.x;  // 2 or 1
      int local = 0;
      for (int u = 0; u < per; ++u) local += (int)hist[0][nb - 1 - (threadIdx.x * per + u)];
      int tot;
      int excl = block_excl_scan(local, warp_buf, &tot);  // keys in bins above my first bin
      int acc = excl;
      for (int u = 0; u < per; ++u) {
        const int b = nb - 1 - (threadIdx.x * per + u);
        const int h = (int)hist[0][b];
        if (acc < need && need <= acc + h) {
          s_digit = (uint32_t)b;
          s_need = need - acc;
        }
        acc += h;
      }
      __syncthreads();
      prefix |= s_digit << shift;
      pmask |= (uint32_t)(nb - 1) << shift;
      need = s_need;
      __syncthreads();
    }
  }
  *need_out = need;
  return prefix;
}

// Top-k of `rows` dense rows: row r is S[r * ld .. r * ld + N).  Scores are
// float (float paths) or int32 (uint8 path).  Output row-major [rows x k].
// only: NULL, or [rows] flags: rows whose flag is 0 are skipped.
template <typename ST>
__global__ void __launch_bounds__(kTopkThreads) topk_dense_rows_kernel(const ST* __restrict__ S, int64_t ld,
                                                                       int64_t N, int k,
                                                                       int32_t* __restrict__ out_ids,
                                                                       ST* __restrict__ out_scores,
                                                                       const uint32_t* __restrict__ only) {
  // the histograms and, after the radix passes, the k candidates share storage
  __shared__ uint32_t smem_raw[kHistCopies * 2048];
  static_assert(2 * GS_MAX_K <= kHistCopies * 2048, "candidates must fit in the histogram storage");
  uint32_t(*hist)[2048] = reinterpret_cast<uint32_t(*)[2048]>(smem_raw);
  uint32_t* cand_key = smem_raw;
  int32_t* cand_id = reinterpret_cast<int32_t*>(smem_raw + GS_MAX_K);
  __shared__ int warp_buf[32];
  __shared__ uint32_t s_digit;
  __shared__ int s_need;
  __shared__ int s_gt;

  const int row = blockIdx.x;
  if (only && __ldcg(only + row) == 0u) return;
  const ST* __restrict__ r = S + (int64_t)row * ld;

  int need = k;
  const uint32_t prefix = radix_kth_key(r, N, k, hist, warp_buf, &s_digit, &s_need, &need);
  // prefix is now the k-th largest key; `need` ties at it are taken (lowest ids)
  const uint32_t theta = prefix;
  const int n_gt = k - need;
  if (threadIdx.x == 0) s_gt = 0;
  __syncthreads();
  int ties_taken = 0;
  __syncthreads();  // histogram storage becomes the candidate arrays
  const int64_t iters = (N + blockDim.x - 1) / blockDim.x;
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t i = it * blockDim.x + threadIdx.x;
    int tie = 0;
    if (i < N) {
      const uint32_t key = score_key(r[i]);
      if (key > theta) {
        const int slot = atomicAdd(&s_gt, 1);
        if (slot < n_gt) {
          cand_key[slot] = key;
          cand_id[slot] = (int32_t)i;
        }
      } else if (key == theta) {
        tie = 1;
      }
    }
    if (ties_taken < need) {  // block-uniform
      int tot;
      const int rank = ties_taken + block_excl_scan(tie, warp_buf, &tot);
      if (tie && rank < need) {
        cand_key[n_gt + rank] = theta;
        cand_id[n_gt + rank] = (int32_t)i;
      }
      ties_taken += tot;
    }
  }
  __syncthreads();
  int n_pad = 1;
  while (n_pad < k) n_pad <<= 1;
  for (int i = k + threadIdx.x; i < n_pad; i += blockDim.x) {
    cand_key[i] = 0u;
    cand_id[i] = 0x7fffffff;
  }
  bitonic_sort_desc(cand_key, cand_id, n_pad);
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    out_ids[(int64_t)row * k + j] = cand_id[j];
    out_scores[(int64_t)row * k + j] = key_to_score<ST>(cand_key[j]);
  }
}

// A lower bound of the k-th largest score of each of `rows` dense rows (raw
// score bits).  Float scores: the k-th largest key with its 10 low bits
// cleared, the lower edge of its bin after two radix passes (22 key bits);
// the bin is 2^-13 of the score wide, so it admits few extra candidates.
// Integer scores: the k-th largest score itself (three passes).  The
// doc-tiled path needs only a lower bound from its sample.
template <typename ST>
__global__ void __launch_bounds__(kTopkThreads) kth_score_rows_kernel(const ST* __restrict__ S, int64_t ld, int64_t N,
                                                                      int k, uint32_t* __restrict__ out_bits) {
  __shared__ uint32_t hist[kHistCopies][2048];
  __shared__ int warp_buf[32];
  __shared__ uint32_t s_digit;
  __shared__ int s_need;
  int need = k;
  const int passes = std::is_same<ST, float>::value ? 2 : 3;
  const uint32_t key =
      radix_kth_key(S + (int64_t)blockIdx.x * ld, N, k, hist, warp_buf, &s_digit, &s_need, &need, passes);
  if (threadIdx.x == 0) {
    const ST v = key_to_score<ST>(key);
    uint32_t bits;
    memcpy(&bits, &v, 4);
    out_bits[blockIdx.x] = bits;
  }
}

}  // namespace gs
