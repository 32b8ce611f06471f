// Query order of a doc-tiled batch: queries whose sparse-tail terms overlap
// are placed in the same group of G queries.
//
// The doc-tiled kernel reads each tile segment of a group's distinct tail
// terms once and adds every posting into all of the group's queries holding
// the term (the batched scatter-add of Sec. 4.1 Eq. 4, with the shared-memory
// accumulation of the hybrid kernel, Sec. 8 future work 1).  A term shared by
// queries of one group is read once for all of them; the same term spread over
// several groups is read once per group.  Regrouping the batch so that queries
// sharing long tail lists sit together therefore cuts the postings the tail
// loads and the per-tile segment planning, while every query's score row and
// top-k stay exactly what they are in the caller's order: the search runs on
// the regrouped batch and writes each result row at its query's own position.
//
// The grouping is a parallel greedy clustering, one CTA per block of at most
// 512 queries and 32 groups (whole groups):
//  - each query keeps its kOrdM tail terms (outside the dense head) with the
//    longest posting lists; a term weighs its list length, the postings a
//    group saves per tile when it shares the term;
//  - queries are ranked by (longest tail list, its term, second longest);
//    group g starts from the query of rank g G, which spreads the seeds over
//    the batch's term space;
//  - the affinity of a free query to a group is the weight of its kept terms
//    inside the group's term set (a 2^13-bit hashed bitmap; a hash collision
//    only misjudges an affinity).  It is kept up to date: when a term enters a
//    group's set, every query holding it (an inverted table from term hash to
//    (query, slot)) gains the term's weight for that group;
//  - in each round every group that still has room proposes its free query of
//    highest affinity; a query proposed by several groups joins the one that
//    weighs it most (ties: the lower group), the others propose again next
//    round;
//  - after G - 1 rounds the free queries fill the open slots in rank order.
// A batch whose row pointer is not a valid CSR keeps the caller's order (a
// verbatim copy), so the search flags and treats it exactly as before.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "gs_doctiled.cuh"
#include "gs_topk.cuh"

namespace gs {
namespace {

constexpr int kOrdThreads = 1024;
constexpr int kOrdMinGroup = 8;    // smaller groups are not regrouped
constexpr int kOrdQueries = 512;   // queries ordered by one CTA (whole groups) ...
constexpr int kOrdMaxGroups = 32;  // ... in at most this many groups
constexpr int kOrdM = 8;           // tail terms per query that count
constexpr int kOrdBitsLog = 13;    // term hashes of 13 bits
constexpr int kOrdBuckets = 1 << kOrdBitsLog;
constexpr int kOrdWords = kOrdBuckets / 32;

// Knuth's multiplicative hash (the golden-ratio constant 2^32 / phi)
__device__ __forceinline__ uint32_t term_hash(int32_t t) {
  return ((uint32_t)t * 2654435761u) >> (32 - kOrdBitsLog);
}

// (affinity, group) -> one word whose maximum is the highest affinity, then the lowest group
__device__ __forceinline__ unsigned long long claim_word(float s, int g) {
  return ((unsigned long long)__float_as_uint(s) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)g);
}

// queries ordered together: whole groups, at most kOrdQueries queries and kOrdMaxGroups groups
__host__ __device__ constexpr int order_block(int G) {
  return (kOrdQueries / G < kOrdMaxGroups ? kOrdQueries / G : kOrdMaxGroups) * G;
}

size_t order_smem_bytes(int nb, int G) {
  const size_t ngm = (size_t)(nb / G);
  return (size_t)nb * (8 + 8 + 4 * kOrdM + 2 * kOrdM + 2 * kOrdM + 4 * 3) + ngm * (kOrdWords + nb) * 4 +
         (size_t)(kOrdBuckets + 1) * 4;
}

__global__ void __launch_bounds__(kOrdThreads) dt_order_kernel(
    const int32_t* __restrict__ q_indptr, const int32_t* __restrict__ q_terms, const float* __restrict__ q_w,
    int32_t B, int32_t q_nnz, int G, int32_t V, const int32_t* __restrict__ head_slot,
    const int32_t* __restrict__ term_len, int32_t* __restrict__ o_indptr, int32_t* __restrict__ o_terms,
    float* __restrict__ o_w, int32_t* __restrict__ perm) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int s_cnt[kOrdMaxGroups], s_prop[kOrdMaxGroups], s_open[kOrdMaxGroups + 1];
  __shared__ float s_pscore[kOrdMaxGroups];
  __shared__ int warp_buf[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = order_block(G);
  const int base = blockIdx.x * nb;
  const int n = min(nb, B - base);
  const int ngb = (n + G - 1) / G;

  // the row pointer is device data: a batch that is not a valid CSR keeps its order
  int bad = 0;
  for (int q = threadIdx.x; q < B; q += blockDim.x) bad |= q_indptr[q + 1] < q_indptr[q];
  if (threadIdx.x == 0) bad |= q_indptr[0] != 0 || q_indptr[B] > q_nnz || q_indptr[B] < 0;
  if (__syncthreads_or(bad)) {
    for (int i = base + (int)threadIdx.x; i < base + n; i += blockDim.x) {
      o_indptr[i] = q_indptr[i];
      perm[i] = i;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) o_indptr[B] = q_indptr[B];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < q_nnz; e += (int64_t)gridDim.x * blockDim.x) {
      o_terms[e] = q_terms[e];
      o_w[e] = q_w[e];
    }
    return;
  }

  const int ngm = nb / G;  // groups of a full block
  unsigned long long* s_key = reinterpret_cast<unsigned long long*>(smem);  // [nb] rank key
  unsigned long long* s_claim = s_key + nb;                                 // [nb] best proposal
  float* s_tw = reinterpret_cast<float*>(s_claim + nb);                     // [M][nb] term weights
  float* s_aff = s_tw + kOrdM * nb;                                         // [ngm][nb] affinities
  uint32_t* s_bm = reinterpret_cast<uint32_t*>(s_aff + ngm * nb);           // [ngm][words] term sets
  uint32_t* s_boff = s_bm + ngm * kOrdWords;                                // [buckets + 1] inverted table
  uint16_t* s_th = reinterpret_cast<uint16_t*>(s_boff + kOrdBuckets + 1);   // [M][nb] term hashes
  uint16_t* s_inv = s_th + kOrdM * nb;                                      // [nb M] (query << 3 | slot)
  int32_t* s_grp = reinterpret_cast<int32_t*>(s_inv + kOrdM * nb);          // [nb] group, -1: free
  int32_t* s_byrank = s_grp + nb;                                           // [nb] query of each rank
  int32_t* s_mem = s_byrank + nb;                                           // [nb] members, group-major

  for (int x = threadIdx.x; x < ngb * kOrdWords; x += blockDim.x) s_bm[x] = 0u;
  for (int x = threadIdx.x; x < ngb * nb; x += blockDim.x) s_aff[x] = 0.f;
  for (int x = threadIdx.x; x <= kOrdBuckets; x += blockDim.x) s_boff[x] = 0u;
  // each query's kOrdM tail terms with the longest lists, and its rank key:
  // an 8-lane quarter of a warp per query, each lane keeping the best kOrdM
  // of its own terms (every 8th entry), merged by kOrdM quarter-wide maxima
  const int sl = lane & 7;
  for (int i0 = 4 * warp; i0 < n; i0 += 4 * (kOrdThreads / 32)) {
    const int i = i0 + (lane >> 3);
    float tw[kOrdM];
    int32_t tt[kOrdM];
#pragma unroll
    for (int j = 0; j < kOrdM; ++j) {
      tw[j] = 0.f;
      tt[j] = -1;
    }
    if (i < n)
      for (int32_t e = q_indptr[base + i] + sl; e < q_indptr[base + i + 1]; e += 8) {
        int32_t t = __ldg(q_terms + e);
        if (t < 0 || t >= V) continue;
        if (head_slot && __ldg(head_slot + t) >= 0) continue;
        float w = (float)__ldg(term_len + t);
        if (!(w > tw[kOrdM - 1])) continue;
#pragma unroll
        for (int j = 0; j < kOrdM; ++j) {  // insertion into the lane's sorted list
          if (w > tw[j]) {
            const float w0 = tw[j];
            const int32_t t0 = tt[j];
            tw[j] = w;
            tt[j] = t;
            w = w0;
            t = t0;
          }
        }
      }
    float w1 = 0.f, w2 = 0.f;
    int32_t t1 = -1;
#pragma unroll
    for (int j = 0; j < kOrdM; ++j) {
      // the quarter's largest remaining weight (ties: the lower lane) leaves its lane's list
      float bw = tw[0];
      int bl = lane;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const float ow = __shfl_xor_sync(0xffffffffu, bw, o);
        const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
        if (ow > bw || (ow == bw && ol < bl)) {
          bw = ow;
          bl = ol;
        }
      }
      const int32_t bt = __shfl_sync(0xffffffffu, tt[0], bl);
      if (lane == bl) {
#pragma unroll
        for (int x = 0; x + 1 < kOrdM; ++x) {
          tw[x] = tw[x + 1];
          tt[x] = tt[x + 1];
        }
        tw[kOrdM - 1] = 0.f;
        tt[kOrdM - 1] = -1;
      }
      if (sl == 0 && i < n) {
        s_tw[j * nb + i] = bw;
        s_th[j * nb + i] = (uint16_t)(bw > 0.f ? term_hash(bt) : 0u);
      }
      if (j == 0) {
        w1 = bw;
        t1 = bw > 0.f ? bt : -1;
      }
      if (j == 1) w2 = bw;
    }
    if (sl == 0 && i < n) {
      const uint32_t d1 = min((uint32_t)w1, 0xFFFFFFu), d2 = min((uint32_t)w2, 0x7FFFFFu);
      s_key[i] = ((unsigned long long)(0xFFFFFFu - d1) << 40) | ((unsigned long long)((uint32_t)t1 & 0x1FFFFu) << 23) |
                 (unsigned long long)(0x7FFFFFu - d2);
      s_grp[i] = -1;
      s_claim[i] = 0ull;
    }
  }
  __syncthreads();
  // inverted table: bucket h lists the (query, slot) pairs whose term hashes
  // to h, at [h ? s_boff[h - 1] : 0, s_boff[h]) once filled
  for (int x = threadIdx.x; x < n * kOrdM; x += blockDim.x) {
    const int j = x / n, i = x - j * n;
    if (s_tw[j * nb + i] > 0.f) atomicAdd(&s_boff[s_th[j * nb + i]], 1u);
  }
  __syncthreads();
  {
    constexpr int kPer = kOrdBuckets / kOrdThreads;
    uint32_t c[kPer], loc = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      c[u] = s_boff[threadIdx.x * kPer + u];
      loc += c[u];
    }
    int tot;
    uint32_t run = (uint32_t)block_excl_scan((int)loc, warp_buf, &tot);
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      s_boff[threadIdx.x * kPer + u] = run;  // the bucket's start; the fill advances it to its end
      run += c[u];
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < n * kOrdM; x += blockDim.x) {
    const int j = x / n, i = x - j * n;
    if (s_tw[j * nb + i] > 0.f) s_inv[atomicAdd(&s_boff[s_th[j * nb + i]], 1u)] = (uint16_t)(i << 3 | j);
  }
  // rank of every query by its key
  if ((int)threadIdx.x < n) {
    const int i = threadIdx.x;
    const unsigned long long ki = s_key[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const unsigned long long kj = s_key[j];
      r += (kj < ki) || (kj == ki && j < i);
    }
    s_byrank[r] = i;
  }
  __syncthreads();

  // query q joins group g (the group's warp): each of its kept terms new to the
  // group's set enters it, and every query holding that term gains its weight
  auto join = [&](int g, int q) {
    uint32_t* bm = s_bm + g * kOrdWords;
    float* aff = s_aff + g * nb;
    for (int j = 0; j < kOrdM; ++j) {
      if (!(s_tw[j * nb + q] > 0.f)) break;  // kept terms are sorted: the rest are empty
      const uint32_t h = s_th[j * nb + q];
      const bool fresh = !((bm[h >> 5] >> (h & 31)) & 1u);
      __syncwarp();
      if (!fresh) continue;
      if (lane == 0) bm[h >> 5] |= 1u << (h & 31);
      const uint32_t b0 = h ? s_boff[h - 1] : 0u, b1 = s_boff[h];
      for (uint32_t e = b0 + lane; e < b1; e += 32) {
        const uint32_t v = s_inv[e];
        const int qq = (int)(v >> 3), jj = (int)(v & 7u);
        atomicAdd(&aff[qq], s_tw[jj * nb + qq]);
      }
      __syncwarp();
    }
  };
  // seeds: group g starts from the query of rank g G
  if (warp < ngb) {
    const int g = warp, q = s_byrank[g * G];
    if (lane == 0) {
      s_grp[q] = g;
      s_mem[g * G] = q;
      s_cnt[g] = 1;
    }
    join(g, q);
  }
  __syncthreads();

  for (int round = 1; round < G; ++round) {
    // proposals: warp g serves group g
    if (warp < ngb) {
      const int g = warp;
      const int cap = min(G, n - g * G);
      float best_s = -1.f;
      int best_q = -1;
      if (s_cnt[g] < cap) {
        const float* aff = s_aff + g * nb;
        for (int q = lane; q < n; q += 32) {
          if (s_grp[q] >= 0) continue;
          const float sc = aff[q];
          if (sc > best_s) {  // a lane's queries rise: the first maximum is its lowest
            best_s = sc;
            best_q = q;
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, best_s, o);
        const int oq = __shfl_xor_sync(0xffffffffu, best_q, o);
        if (oq >= 0 && (os > best_s || (os == best_s && (best_q < 0 || oq < best_q)))) {
          best_s = os;
          best_q = oq;
        }
      }
      if (lane == 0) {
        s_prop[g] = best_q;
        s_pscore[g] = best_s;
        if (best_q >= 0) atomicMax(&s_claim[best_q], claim_word(best_s, g));
      }
    }
    __syncthreads();
    // every claimed query joins the group that weighs it most
    if (warp < ngb) {
      const int g = warp, q = s_prop[g];
      if (q >= 0 && s_claim[q] == claim_word(s_pscore[g], g)) {
        if (lane == 0) {
          s_grp[q] = g;
          s_mem[g * G + s_cnt[g]] = q;
          s_cnt[g] += 1;
        }
        join(g, q);
      }
    }
    __syncthreads();
    int proposed = 0;
    if ((int)threadIdx.x < ngb) {
      const int q = s_prop[threadIdx.x];
      if (q >= 0) {
        s_claim[q] = 0ull;
        proposed = 1;
      }
    }
    if (!__syncthreads_or(proposed)) break;
  }

  // free queries, in rank order, take the open slots in group order
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int g = 0; g < ngb; ++g) {
      s_open[g] = acc;
      acc += min(G, n - g * G) - s_cnt[g];
    }
    s_open[ngb] = acc;
  }
  __syncthreads();
  const int rq = (int)threadIdx.x < n ? s_byrank[threadIdx.x] : -1;
  const int is_free = rq >= 0 && s_grp[rq] < 0;
  int n_free;
  const int fidx = block_excl_scan(is_free, warp_buf, &n_free);
  if (is_free) {
    int g = 0;
    while (g + 1 < ngb && s_open[g + 1] <= fidx) ++g;
    s_mem[g * G + s_cnt[g] + (fidx - s_open[g])] = rq;
  }
  __syncthreads();

  // position p of the block (group-major) holds query base + s_mem[p]
  int len = 0;
  if ((int)threadIdx.x < n) {
    const int o = base + s_mem[threadIdx.x];
    len = q_indptr[o + 1] - q_indptr[o];
    perm[base + threadIdx.x] = o;
  }
  int tot;
  const int off = block_excl_scan(len, warp_buf, &tot);
  const int32_t e_base = q_indptr[base];
  if ((int)threadIdx.x < n) {
    o_indptr[base + threadIdx.x] = e_base + off;
    s_grp[threadIdx.x] = off;  // group membership is no longer needed: output offsets
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) o_indptr[B] = q_indptr[B];
  __syncthreads();
  for (int p = warp; p < n; p += kOrdThreads / 32) {
    const int o = base + s_mem[p];
    const int32_t a = q_indptr[o], cnt = q_indptr[o + 1] - a, d = e_base + s_grp[p];
    for (int32_t e = lane; e < cnt; e += 32) {
      o_terms[d + e] = __ldg(q_terms + a + e);
      o_w[d + e] = __ldg(q_w + a + e);
    }
  }
}

}  // namespace

bool dt_order_used(int32_t B, int G, int64_t N, const gs_search_opts* opts) {
  const int mode = opts ? opts->query_order : 0;
  if (mode < 0 || G < kOrdMinGroup || B < 2 * G) return false;
  if (mode > 0) return true;
  // default: regroup when the main pass is long enough for its saving (about 4%
  // of ~4.6 ns per query and document on GB300) to exceed 1.5 times the cost of
  // the regrouping (about 40 us + 0.18 us per query), both measured on the
  // synthetic MS MARCO-like workload (1M and 8.84M documents, batches 32 to 500)
  const double gain_ms = 1.85e-10 * (double)B * (double)N;
  const double cost_ms = 0.04 + 1.8e-4 * (double)B;
  return B >= 4 * G && gain_ms > 1.5 * cost_ms;
}

gs_status dt_order_prepare_device() {
  static std::mutex mu;
  static bool done[128] = {};
  int dev = 0;
  GS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 128) return GS_ERR_UNSUPPORTED;
  if (!done[dev]) {
    size_t most = 0;
    for (int G = kOrdMinGroup; G <= kOrdQueries; ++G) most = std::max(most, order_smem_bytes(order_block(G), G));
    GS_CUDA_TRY(cudaFuncSetAttribute(dt_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most));
    done[dev] = true;
  }
  return GS_OK;
}

gs_status dt_order(const gs_index* ix, const int32_t* q_indptr, const int32_t* q_terms, const float* q_w, int32_t B,
                   int32_t q_nnz, int G, const int32_t* head_slot, int32_t* o_indptr, int32_t* o_terms, float* o_w,
                   int32_t* perm, cudaStream_t s) {
  if (G < kOrdMinGroup) return GS_ERR_INVALID_ARG;
  const int nb = order_block(G);
  const int blocks = (B + nb - 1) / nb;
  dt_order_kernel<<<blocks, kOrdThreads, order_smem_bytes(nb, G), s>>>(
      q_indptr, q_terms, q_w, B, q_nnz, G, ix->V, head_slot, ix->term_len, o_indptr, o_terms, o_w, perm);
  GS_LAUNCH_CHECK();
  return GS_OK;
}

}  // namespace gs
