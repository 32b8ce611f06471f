// Doc-tiled scoring with a sampled threshold (the hybrid kernel the paper
// proposes as future work 1, Sec. 8: scatter-add work efficiency with
// shared-memory accumulation), designed for sm_103a.
//
// The queries of a batch form groups of G consecutive queries; the documents
// form tiles of T consecutive ids.  A CTA owns one group and a run of tiles and
// keeps the G x T block of score rows of its current tile in shared memory.
// Sparse tail: for every distinct term of the group outside the dense head it
// reads the segment of the term's posting list that falls inside the tile (the
// segment table of the index gives its bounds, lists being doc-sorted, Sec. 3.2)
// once, 32 postings per warp step, and adds w * x into the rows of every query
// of the group holding the term (shared-memory reductions, no global atomics;
// integer reductions in fixed point where a bound on the tail score allows).
// Padding (doc -1) lies outside every segment.  Dense head: the most frequent
// terms' rows are multiplied densely (CUDA-core FMAs or tensor-core MMAs).
//
// Exact top-k without dense rows: every R-th full tile is a sample tile.  The
// sample tiles are scored first and written out; theta_q, the k-th largest
// sample score of query q (rounded down to 22 key bits for float scores), is a
// lower bound of its k-th largest score over all documents.  The remaining
// tiles are then scored, and every document with score > theta_q is appended
// to a per-query candidate list; documents equal to theta_q set a bit in a
// per-query tie bitmap.  A final kernel per query returns the top-k of the
// candidates by (score desc, id asc), taking the lowest-id ties when fewer
// than k candidates exceed theta_q.  Every document's score is computed
// exactly once, so the bound holds exactly.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "gs_doctiled.cuh"
#include "gs_tc05.cuh"
#include "gs_topk.cuh"

namespace gs {
namespace {

constexpr int kDtThreads = 512;              // two CTAs per SM (64 registers each)
constexpr int kDtMaxAccBytes = 64 * 1024;    // G x T accumulators
constexpr int kEntCap = 1280;                // query entries staged in shared memory (10 KB)
constexpr int kItemCap = 4608;               // (term, 128-posting chunk) items per term batch (9 KB)
constexpr int kTinySeg = 32;                 // segments shorter than this are packed, not itemised
constexpr int kChunkCap = kDtThreads * kTinySeg / 32 + 1;  // packed 32-posting chunks per term batch
constexpr int kMaxGroup = 64;                // queries per group (thresholds kept in shared memory)
constexpr int kHeadG = 16;                   // queries per group when the dense head is used
constexpr int kDefaultGroup = 16;
constexpr int kDefaultSampleStride = 64;
// dense head kinds: none, CUDA-core FMAs, tensor-core MMAs (warp-level
// mma.sync), tensor-memory MMAs (tcgen05, FP32 impacts)
enum { kHeadNone = 0, kHeadFma = 1, kHeadTensor = 2, kHeadTc05 = 3 };
constexpr int kTc05MaxRows = 24;     // head rows the tensor-memory head takes (3 k-steps of 8)
constexpr uint32_t kTc05Cols = 256;  // tensor-memory columns per CTA (two CTAs per SM)
constexpr uint32_t kTc05WaitTries = 1u << 22;

struct DtConfig {
  int G = 0, T = 0, m = 0, R = 0;  // R = 0: no sampling
  int H = 0;                        // dense head terms used (0: none)
  int HK = kHeadNone;               // how the head is computed
  int ng = 0, nt = 0, n_sample = 0;
  int64_t sample_docs = 0;
  int64_t cap = 0;
  int64_t bm_words = 0;
  bool order = false;  // the batch is regrouped by shared tail terms (gs_order.cu)
};

gs_status dt_config(const gs_index* ix, int B, int k, const gs_search_opts* opts, DtConfig* c) {
  if (!ix->seg) return GS_ERR_UNSUPPORTED;
  c->T = (opts && opts->tile_docs > 0) ? opts->tile_docs : ix->tile_docs;
  // a power of two; at most 64 chunks of 128 documents per row
  if (c->T % ix->tile_docs != 0 || (c->T & (c->T - 1)) != 0 || c->T > 8192) return GS_ERR_INVALID_ARG;
  c->m = c->T / ix->tile_docs;
  int G = (opts && opts->group_queries > 0) ? opts->group_queries : kDefaultGroup;
  // the dense head serves groups of kHeadG queries: CUDA-core FMAs (use_head
  // 1, and FP32 impacts by default), warp-level tensor-core MMAs (use_head 2,
  // and the other impacts by default) or tensor-memory MMAs (use_head 3, FP32
  // impacts, at most 24 head rows); use_head < 0 turns it off
  const int use_head = opts ? opts->use_head : 0;
  if (use_head > 3) return GS_ERR_INVALID_ARG;
  const bool head = ix->head_H > 0 && G == kHeadG && use_head >= 0;
  // the tensor-memory head (use_head 3): FP32 impacts, at most 24 head rows
  if (head && use_head == 3 && (ix->impact != GS_IMPACT_F32 || ix->head_H > kTc05MaxRows)) return GS_ERR_UNSUPPORTED;
  c->HK = !head ? kHeadNone
                : (use_head == 1 ? kHeadFma
                                 : (use_head == 2 ? kHeadTensor
                                                  : (use_head == 3 ? kHeadTc05
                                                                   : (ix->impact == GS_IMPACT_F32 ? kHeadFma
                                                                                                  : kHeadTensor))));
  c->H = head ? ix->head_H : 0;
  G = head ? kHeadG : std::min(std::min(G, B), kMaxGroup);
  if ((int64_t)G * c->T * 4 > kDtMaxAccBytes) {
    if (opts && opts->group_queries > 0) return GS_ERR_INVALID_ARG;
    G = std::max(1, kDtMaxAccBytes / (c->T * 4));
  }
  c->G = G;
  c->ng = (B + G - 1) / G;
  c->nt = (int)((ix->N + c->T - 1) / c->T);
  const int nt_full = (int)(ix->N / c->T);
  int R = (opts && opts->sample_stride > 0) ? opts->sample_stride : kDefaultSampleStride;
  if (opts && opts->sample_stride == 1) R = 0;  // caller asked for no sampling
  // the sample must hold at least 2k documents
  while (R > 1 && (int64_t)((nt_full + R - 1) / R) * c->T < 2 * (int64_t)k) R /= 2;
  if (R >= 1 && (int64_t)((nt_full + R - 1) / R) * c->T < (int64_t)k) R = 0;
  if (R == 1 && nt_full == c->nt) R = 0;  // everything would be sample: score once, no threshold
  c->R = R;
  c->n_sample = R > 0 ? (nt_full + R - 1) / R : 0;
  c->sample_docs = (int64_t)c->n_sample * c->T;
  const int64_t n_round = (ix->N + 255) / 256 * 256;
  c->cap = R > 0 ? std::min<int64_t>(n_round, (4 * (int64_t)k * R + 4096 + 255) / 256 * 256) : n_round;
  c->bm_words = (ix->N + 31) / 32;
  c->order = dt_order_used(B, c->G, ix->N, opts);
  return GS_OK;
}

struct DtPlan {
  uint32_t* cnt;      // [ng][V]
  int32_t* u_terms;   // group g at q_indptr[gG]
  int32_t* u_ptr;     // group g at q_indptr[gG] + g
  int32_t* n_u;       // [ng]
  uint2* ent;         // [q_nnz] (query within group, weight bits)
  uint32_t* samp;     // [B][sample_docs]
  uint32_t* theta;    // [B] lower bound of the k-th largest sample score (raw bits)
  uint2* cand;        // [B][cap] (key, doc)
  uint32_t* cand_cnt; // [B]; the cleared block [B cand_cnt][B q_over][ng g_mark][n_groups]
  uint32_t* q_over;   // [B] 1: the query's candidate list overflowed
  uint32_t* g_mark;   // [ng] 1: the group is on the recovery list
  uint32_t* n_ovg;    // groups on the recovery list
  int32_t* ov_groups; // [ng] the recovery list
  uint32_t* ov_prefix;// [B] resolved key bits of the exact k-th score
  int32_t* ov_need;   // [B] documents at the current prefix still to take
  uint32_t* ov_theta; // [B] the exact k-th score (raw bits)
  uint32_t* ov_hist;  // [B][2048] digit histogram
  size_t zero_bytes;  // bytes of the cleared block
  uint32_t* tiebm;    // [B][bm_words]
  uint32_t* headw;    // [ng][H][kHeadG] head weights (float or int bits)
  int32_t* head_act;  // [ng][H] head rows with a non-zero weight
  int32_t* head_nact; // [ng]
  int32_t* fixp;      // [ng] 1: fixed-point tail
  int32_t* qscale;    // [B] S_q of the fixed-point tail
  int32_t* o_indptr;  // regrouped batch (c.order): query CSR [B + 1], [q_nnz], [q_nnz]
  int32_t* o_terms;
  float* o_w;
  int32_t* perm;      // [B] the caller's query at each position of the regrouped batch
};

DtPlan carve_dt(void* ws, const gs_index* ix, int B, int64_t q_nnz, int k, const DtConfig& c, size_t* bytes) {
  Carver cv(ws);
  DtPlan p{};
  p.cnt = cv.take<uint32_t>((size_t)c.ng * ix->V);
  p.u_terms = cv.take<int32_t>(q_nnz + 1);
  p.u_ptr = cv.take<int32_t>(q_nnz + c.ng + 1);
  p.n_u = cv.take<int32_t>(c.ng);
  p.ent = cv.take<uint2>(q_nnz + 1);
  p.samp = cv.take<uint32_t>((size_t)B * std::max<int64_t>(c.sample_docs, 1));
  p.theta = cv.take<uint32_t>(B);
  p.cand = cv.take<uint2>((size_t)B * c.cap);
  p.zero_bytes = sizeof(uint32_t) * (2 * (size_t)B + c.ng + 1);
  p.cand_cnt = cv.take<uint32_t>(2 * (size_t)B + c.ng + 1);
  p.q_over = p.cand_cnt ? p.cand_cnt + B : nullptr;
  p.g_mark = p.cand_cnt ? p.q_over + B : nullptr;
  p.n_ovg = p.cand_cnt ? p.g_mark + c.ng : nullptr;
  p.ov_groups = cv.take<int32_t>(c.ng);
  p.ov_prefix = cv.take<uint32_t>(B);
  p.ov_need = cv.take<int32_t>(B);
  p.ov_theta = cv.take<uint32_t>(B);
  p.ov_hist = cv.take<uint32_t>((size_t)B * 2048);
  p.tiebm = cv.take<uint32_t>((size_t)B * c.bm_words);
  p.headw = cv.take<uint32_t>((size_t)c.ng * std::max(c.H, 1) * kHeadG);
  p.head_act = cv.take<int32_t>((size_t)c.ng * std::max(c.H, 1));
  p.head_nact = cv.take<int32_t>(c.ng);
  p.fixp = cv.take<int32_t>(c.ng);
  p.qscale = cv.take<int32_t>(B);
  if (c.order) {
    p.o_indptr = cv.take<int32_t>((size_t)B + 1);
    p.o_terms = cv.take<int32_t>(q_nnz + 1);
    p.o_w = cv.take<float>(q_nnz + 1);
    p.perm = cv.take<int32_t>(B);
  }
  *bytes = cv.size();
  return p;
}

__device__ __forceinline__ int ub_i32(const int32_t* a, int n, int32_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One CTA per group: distinct terms of the group (in term order) and, per
// term, the (query-in-group, weight) entries; invalid pairs are skipped.
__global__ void __launch_bounds__(1024) dt_prep_kernel(const int32_t* __restrict__ q_indptr,
                                                       const int32_t* __restrict__ q_terms,
                                                       const float* __restrict__ q_w, int32_t B, int32_t q_nnz,
                                                       int G, int32_t V,
                                                       int impact, uint32_t* __restrict__ cnt_all,
                                                       int32_t* __restrict__ u_terms, int32_t* __restrict__ u_ptr,
                                                       int32_t* __restrict__ n_u, uint2* __restrict__ ent,
                                                       const int32_t* __restrict__ head_slot, int H,
                                                       uint32_t* __restrict__ headw, int32_t* __restrict__ head_act,
                                                       int32_t* __restrict__ head_nact,
                                                       const float* __restrict__ max_abs, int32_t* __restrict__ fixp,
                                                       int32_t* __restrict__ qscale, uint32_t* flags) {
  __shared__ int warp_buf[32];
  __shared__ float s_U[kMaxGroup];  // per query: sum over tail entries of |w| max|x|
  __shared__ int s_n[kMaxGroup];    // per query: tail entries
  __shared__ int s_ok;
  const int g = blockIdx.x;
  const int q0 = g * G, q1 = min(B, q0 + G);
  uint32_t fl = 0;
  // the query CSR is device data: check it, and keep every access in bounds
  for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    if (q_indptr[q + 1] < q_indptr[q]) fl |= GS_FLAG_BAD_INDPTR;
  }
  if (threadIdx.x == 0 && (q_indptr[0] != 0 || q_indptr[B] > q_nnz || q_indptr[B] < 0)) fl |= GS_FLAG_BAD_INDPTR;
  const int32_t e0 = min(max(q_indptr[q0], 0), q_nnz);
  const int32_t e1 = min(max(q_indptr[q1], e0), q_nnz);
  uint32_t* cnt = cnt_all + (int64_t)g * V;
  for (int t = threadIdx.x; t < V; t += blockDim.x) cnt[t] = 0u;
  uint32_t* hw = headw + (int64_t)g * H * kHeadG;
  for (int i = threadIdx.x; i < H * kHeadG; i += blockDim.x) hw[i] = 0u;
  for (int i = threadIdx.x; i < kMaxGroup; i += blockDim.x) {
    s_U[i] = 0.f;
    s_n[i] = 0;
  }
  if (threadIdx.x == 0) s_ok = impact != GS_IMPACT_U8;
  __syncthreads();
  for (int32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int32_t t = q_terms[e];
    const float w = q_w[e];
    if (t < 0 || t >= V) { fl |= kFlagBadTerm; continue; }
    if (!isfinite(w)) { fl |= kFlagBadWeight; continue; }
    if (H > 0 && __ldg(head_slot + t) >= 0) {  // a head term: dense weight row
      const int ql = min(max(ub_i32(q_indptr + q0, q1 - q0 + 1, e) - 1, 0), q1 - q0 - 1);
      uint32_t* slotp = hw + (int64_t)__ldg(head_slot + t) * kHeadG + ql;
      if (impact == GS_IMPACT_U8) atomicAdd(reinterpret_cast<int32_t*>(slotp), quant_u8(w));
      else atomicAdd(reinterpret_cast<float*>(slotp), w);
      continue;
    }
    atomicAdd(&cnt[t], 1u);
  }
  __syncthreads();
  // distinct terms in increasing id; entry offsets
  int carry_u = 0, carry_e = 0;
  const int ubase = e0, pbase = e0 + g;
  for (int t0 = 0; t0 < V; t0 += blockDim.x) {
    const int t = t0 + threadIdx.x;
    const int c = (t < V) ? (int)__ldcg(&cnt[t]) : 0;
    int tot_u, tot_e;
    const int xu = block_excl_scan(c > 0 ? 1 : 0, warp_buf, &tot_u);
    const int xe = block_excl_scan(c, warp_buf, &tot_e);
    if (c > 0) {
      u_terms[ubase + carry_u + xu] = t;
      u_ptr[pbase + carry_u + xu] = e0 + carry_e + xe;
      cnt[t] = (uint32_t)(e0 + carry_e + xe);  // fill position
    }
    carry_u += tot_u;
    carry_e += tot_e;
  }
  if (threadIdx.x == 0) {
    n_u[g] = carry_u;
    u_ptr[pbase + carry_u] = e0 + carry_e;
  }
  __syncthreads();
  for (int32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int32_t t = q_terms[e];
    const float w = q_w[e];
    if (t < 0 || t >= V || !isfinite(w)) continue;
    if (H > 0 && __ldg(head_slot + t) >= 0) continue;
    const int ql = min(max(ub_i32(q_indptr + q0, q1 - q0 + 1, e) - 1, 0), q1 - q0 - 1);
    const uint32_t pos = atomicAdd(&cnt[t], 1u);
    const uint32_t wb = impact == GS_IMPACT_U8 ? (uint32_t)quant_u8(w) : __float_as_uint(w);
    ent[pos] = make_uint2((uint32_t)ql, wb);
    if (impact != GS_IMPACT_U8) {
      atomicAdd(&s_U[ql], fabsf(w) * __ldg(max_abs + t));
      atomicAdd(&s_n[ql], 1);
    }
  }
  // Fixed-point tail (float impacts): query q's tail products w x are added as
  // integers round(w x 2^S_q).  With U_q >= sum |w| max|x| over its n_q tail
  // entries, 2^S_q <= (2^31 - 2^10 - n_q) / U_q keeps every partial sum inside
  // int32, and the rounding error n_q 2^-(S_q + 1) must stay within 0.9e-6 (the
  // tolerance's absolute term); otherwise the group keeps float reductions.
  __syncthreads();
  const int gq = q1 - q0;
  if ((int)threadIdx.x < gq && impact != GS_IMPACT_U8) {
    const float U = s_U[threadIdx.x] * (1.0f + 1.0f / 1024.0f);  // margin for the float sum of U
    const int n = s_n[threadIdx.x];
    int S = 60;
    if (n > 0) {
      S = (int)floorf(log2f((2147483648.0f - 1024.0f - (float)n) / U));
      S = max(min(S, 60), -60);
      // the bound used 2^S <= (2^31 - 2^10 - n) / U: step down if log2f rounded up
      while (S > -60 && ldexpf(U, S) > 2147483648.0f - 1024.0f - (float)n) --S;
      if ((float)n * ldexpf(1.0f, -(S + 1)) > 0.9e-6f) s_ok = 0;
    }
    qscale[q0 + threadIdx.x] = S;
  }
  __syncthreads();
  if (threadIdx.x == 0) fixp[g] = s_ok;
  // head rows some query of the group uses
  if (H > 0) {
    __syncthreads();
    int used = 0;
    if ((int)threadIdx.x < H)
      for (int q = 0; q < kHeadG; ++q) used |= __ldcg(hw + threadIdx.x * kHeadG + q) != 0u;
    int tot;
    const int x = block_excl_scan(used, warp_buf, &tot);
    if (used) head_act[(int64_t)g * H + x] = (int32_t)threadIdx.x;
    if (threadIdx.x == 0) head_nact[g] = tot;
  }
  if (fl) atomicOr(flags, fl);
}

template <int IMPACT>
__device__ __forceinline__ float load_x(const uint8_t* blk, int lane) {
  if (IMPACT == GS_IMPACT_F32) return __ldg(reinterpret_cast<const float*>(blk + 128) + lane);
  if (IMPACT == GS_IMPACT_F16) return __half2float(__ldg(reinterpret_cast<const __half*>(blk + 128) + lane));
  if (IMPACT == GS_IMPACT_BF16)
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(blk + 128) + lane));
  return (float)__ldg(blk + 128 + lane);
}

// Passes of the tile kernel: the sample tiles, the other tiles (candidates
// above the sampled threshold), and the recovery passes of queries whose
// candidate list overflowed (a persistent grid over their groups, every tile;
// see dt_search).
enum { kModeSample = 0, kModeMain = 1, kModeRecover = 2 };

// State of the exact recovery of overflowed queries (device workspace).
struct DtRecover {
  const int32_t* groups;     // [ng] groups holding an overflowed query
  const uint32_t* n_groups;  // how many
  const uint32_t* q_over;    // [B] 1: the query's top-k is recomputed
  uint32_t* hist;            // [B][2048] digit histogram of the current pass
  const uint32_t* prefix;    // [B] key bits resolved by the earlier passes
  const uint32_t* theta;     // [B] the exact k-th score (raw bits), emission pass
  int pass;                  // 0..2: histogram of key digit `pass`; 3: emission
};

// theta_q: key of the k-th largest sample score (stored as raw score bits)
template <typename AccT>
__device__ __forceinline__ uint32_t theta_key(const uint32_t* theta, int64_t q, int R) {
  if (R <= 0) return 0u;  // no sampling: every document is a candidate
  const uint32_t raw = __ldg(theta + q);
  if (std::is_same<AccT, float>::value) return score_key(__uint_as_float(raw));
  return score_key((int32_t)raw);
}

// TF32 operand: x rounded to 10 explicit mantissa bits (ties away from zero)
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// d += A B for one m16n8k8 tile (TF32 operands, FP32 accumulators)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// one stored impact as FP32 (exact)
template <int IMPACT>
__device__ __forceinline__ float load_impact(const uint8_t* p) {
  if (IMPACT == GS_IMPACT_F32) return __ldg(reinterpret_cast<const float*>(p));
  if (IMPACT == GS_IMPACT_F16) return __half2float(__ldg(reinterpret_cast<const __half*>(p)));
  if (IMPACT == GS_IMPACT_BF16) return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(p)));
  return (float)__ldg(p);
}

// element j (0..3) of four consecutive stored impacts, as TF32 operand bits
// (exact: FP16, BF16 and uint8 values have at most 11 significant bits)
__device__ __forceinline__ float f4_get(const float4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
template <int IMPACT, typename V>
__device__ __forceinline__ uint32_t impact_tf32(V v, int j) {
  if constexpr (IMPACT == GS_IMPACT_U8) {
    return __float_as_uint((float)((v >> (8 * j)) & 0xffu));
  } else {
    const uint32_t w = j < 2 ? v.x : v.y;
    const uint16_t hbits = (uint16_t)(j & 1 ? w >> 16 : w & 0xffffu);
    if (IMPACT == GS_IMPACT_BF16) return (uint32_t)hbits << 16;
    return __float_as_uint(__half2float(__ushort_as_half(hbits)));
  }
}

// Barrier of the 4 warps of warpgroup wg (named barriers 1..4; immediate ids,
// so that the kernel reserves 5 barriers rather than all 16, which would allow
// only one resident CTA per SM).
__device__ __forceinline__ void wg_barrier(int wg) {
  switch (wg) {
    case 0: asm volatile("bar.sync 1, 128;" ::: "memory"); break;
    case 1: asm volatile("bar.sync 2, 128;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 3, 128;" ::: "memory"); break;
    default: asm volatile("bar.sync 4, 128;" ::: "memory"); break;
  }
}

// a score cell of the tail: the float itself, or a fixed-point integer times 2^-S
__device__ __forceinline__ float tail_value(float v, bool fx, float isc) {
  return fx ? (float)__float_as_int(v) * isc : v;
}

// One CTA per (query group, run of tiles_per_cta tiles); per tile a G x T
// score block in shared memory, filled by the sparse tail, the dense head and
// read by the candidate epilogue (sample mode: written to the sample rows).
//
// Tail work items are (term, chunk of 4 posting blocks = 128 postings) pairs
// of the group's distinct terms, handed out dynamically to the 16 warps, two
// at a time.  Lane l of a warp takes posting l of each of the 4 blocks, so the
// 32 lanes of one reduction address 32 distinct documents of one query row
// (consecutive documents for dense terms: few bank conflicts), and every
// loaded posting serves all of the group's queries holding the term.
// Segments shorter than kTinySeg are packed 32 postings per warp step.
template <int IMPACT, int MODE, int HK>
__global__ void __launch_bounds__(kDtThreads, 2) dt_tile_kernel(
    const uint8_t* __restrict__ blocks, const int64_t* __restrict__ term_block, const uint32_t* __restrict__ seg,
    int seg_tiles, int64_t N, const int32_t* __restrict__ q_indptr, int32_t B, int32_t q_nnz, int G, int T,
    int m, int R,
    int ng, int n_sample, const int32_t* __restrict__ u_terms, const int32_t* __restrict__ u_ptr,
    const int32_t* __restrict__ n_u, const uint2* __restrict__ ent, uint32_t* __restrict__ samp,
    int64_t sample_docs, const uint32_t* __restrict__ theta, int k, uint2* __restrict__ cand,
    uint32_t* __restrict__ cand_cnt, int64_t cap, uint32_t* __restrict__ tiebm, int64_t bm_words,
    const uint8_t* __restrict__ head_dense, int64_t head_ld, int H, const uint32_t* __restrict__ headw,
    const int32_t* __restrict__ head_act, const int32_t* __restrict__ head_nact, int tiles_per_cta, int n_tiles,
    const int32_t* __restrict__ fixp, const int32_t* __restrict__ qscale, DtRecover rec,
    uint32_t* __restrict__ flags) {
  using AccT = typename std::conditional<IMPACT == GS_IMPACT_U8, int32_t, float>::type;
  constexpr int bb = block_bytes(IMPACT);
  constexpr bool HEAD = HK != kHeadNone;
  // Recovery passes must score every document identically in each of their
  // four passes: float tails then accumulate exact int64 fixed-point sums
  // (order-independent), integer tails are exact already.
  constexpr bool REC64 = MODE == kModeRecover && IMPACT != GS_IMPACT_U8;
  constexpr int kCell = REC64 ? 8 : 4;  // bytes per tail accumulator
  // dynamic shared memory: [G x T accumulators][staged query entries][item -> term]
  extern __shared__ __align__(16) uint8_t dyn_smem[];
  AccT* acc = reinterpret_cast<AccT*>(dyn_smem);
  uint2* ent_s = reinterpret_cast<uint2*>(dyn_smem + (size_t)G * T * kCell);
  uint16_t* item_term = reinterpret_cast<uint16_t*>(ent_s + kEntCap);
  uint16_t* chunk_j0 = item_term + kItemCap;
  __shared__ const uint8_t* s_p0[kDtThreads];  // first block of the term's segment
  __shared__ int32_t s_off[kDtThreads];         // segment start within that block
  __shared__ int32_t s_len[kDtThreads];         // postings in the segment
  __shared__ int32_t s_item[kDtThreads + 1];
  __shared__ int32_t s_tp[kDtThreads + 1];     // packed position of each short segment
  __shared__ int32_t s_e0[kDtThreads + 1];  // entries of term j: [s_e0[j], s_e0[j + 1])
  __shared__ uint32_t s_theta[kMaxGroup];
  __shared__ uint32_t s_over[MODE == kModeRecover ? kMaxGroup : 1];
  __shared__ float s_sc[kMaxGroup], s_isc[kMaxGroup];  // fixed-point tail: 2^S_q and 2^-S_q
  __shared__ int warp_buf[32];
  __shared__ int s_next;
  // head weights: FMA head W[a][q] (a < nact rows, q < 16 queries);
  // tensor-core head m16n8k8 A fragments [k-step][lane] (high part, low part)
  __shared__ uint4 s_af[HEAD ? (GS_MAX_HEAD_TERMS / 8) * 32 * 2 : 1];
  AccT* s_w = reinterpret_cast<AccT*>(s_af);
  __shared__ int s_tc;  // the head runs on the tensor cores
  // tensor-memory head: the CTA's tensor-memory columns and one MMA-completion
  // barrier per warpgroup (warpgroup w uses columns 64 w .. 64 w + 63)
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar[HK == kHeadTc05 ? 4 : 1];
  __shared__ int32_t s_hact[HEAD ? GS_MAX_HEAD_TERMS : 1];

  __shared__ int32_t s_t[kDtThreads];   // the group's terms (one batch)
  __shared__ int32_t s_tb[kDtThreads];  // and their first index blocks

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t_shift = __ffs(T) - 1;  // T is a power of two: cell i lies in row i >> t_shift
  // Main and sample passes: CTA b scores the run of tiles_per_cta tiles
  // that starts at tile (b / ng) tiles_per_cta, for query group b % ng; the
  // group's data are read once and serve all of them.  Recovery passes: a
  // persistent grid walks the (overflowed group, tile run) units.
  uint32_t tmem = 0, mbar_phase = 0;
  bool tc_ok = true;
  if constexpr (HK == kHeadTc05) {
    if (warp == 0) {
      tc05::alloc(&s_tmem, kTc05Cols);
      tc05::relinquish();
    }
    if (threadIdx.x == 0) {
      for (int i = 0; i < 4; ++i) tc05::mbar_init(&s_mbar[i], 1);
      tc05::mbar_init_fence();
    }
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    tmem = s_tmem;
  }
  int n_units = 1, unit0 = 0, ustep = 1, n_ovg = 1;
  if constexpr (MODE == kModeRecover) {
    n_ovg = (int)__ldcg(rec.n_groups);
    n_units = n_ovg * ((n_tiles + tiles_per_cta - 1) / tiles_per_cta);
    unit0 = blockIdx.x;
    ustep = gridDim.x;
  }
  for (int unit = unit0; unit < n_units; unit += ustep) {
    int g, tile_begin;
    if constexpr (MODE == kModeRecover) {
      __syncthreads();  // the previous unit's shared state is no longer read
      g = __ldcg(rec.groups + unit % n_ovg);
      tile_begin = (unit / n_ovg) * tiles_per_cta;
    } else {
      g = blockIdx.x % ng;
      tile_begin = (blockIdx.x / ng) * tiles_per_cta;
    }
    const int tile_end = min(tile_begin + tiles_per_cta, n_tiles);
    const int q0 = g * G;
    const int gq = min(G, B - q0);

    if (MODE == kModeMain)
      for (int i = threadIdx.x; i < gq; i += blockDim.x) s_theta[i] = R > 0 ? __ldg(theta + q0 + i) : 0u;
    if constexpr (MODE == kModeRecover) {
      // histogram passes: the key prefix resolved so far; emission: theta
      for (int i = threadIdx.x; i < gq; i += blockDim.x) {
        s_over[i] = __ldcg(rec.q_over + q0 + i);
        s_theta[i] = __ldcg((rec.pass < 3 ? rec.prefix : rec.theta) + q0 + i);
      }
    }
    const int32_t ebase = min(max(q_indptr[q0], 0), q_nnz);
    const int nterm = n_u[g];
    const int32_t* ut = u_terms + ebase;
    const int32_t* up = u_ptr + ebase + g;
    // fixed-point tail (float impacts, groups whose bound allows it): staged
    // weights carry the query's scale 2^S_q, rows hold integers until the head
    // phase (or a conversion pass) turns them into floats
    // Recovery (float impacts): int64 fixed point with scale 2^(S_q + 30):
    // |w x| 2^(S_q + 30) <= 2^61 per product and per sum (S_q bounds the tail
    // score by 2^31), so no sum overflows and each product is rounded to
    // 2^-(S_q + 31), far inside the tolerance.
    const bool fx = !REC64 && IMPACT != GS_IMPACT_U8 && __ldg(fixp + g) != 0;
    const bool scaled = fx || REC64;
    if (scaled)
      for (int i = threadIdx.x; i < gq; i += blockDim.x) {
        const int S = __ldg(qscale + q0 + i) + (REC64 ? 30 : 0);
        s_sc[i] = ldexpf(1.0f, S);
        s_isc[i] = ldexpf(1.0f, -S);
      }
    __syncthreads();
    // the group's (query, weight) entries, staged with the query's row byte offset
    const int32_t ent_lo = nterm > 0 ? __ldg(up) : 0;
    const int32_t ent_hi = nterm > 0 ? __ldg(up + nterm) : 0;
    const bool staged = (ent_hi - ent_lo) <= kEntCap;
    const uint32_t row_bytes = (uint32_t)T * kCell;
    if (staged)
      for (int i = threadIdx.x; i < ent_hi - ent_lo; i += blockDim.x) {
        const uint2 E = __ldg(ent + ent_lo + i);
        ent_s[i] = make_uint2(E.x * row_bytes, scaled ? __float_as_uint(__uint_as_float(E.y) * s_sc[E.x]) : E.y);
      }
    const uint32_t acc_s = (uint32_t)__cvta_generic_to_shared(acc);
    // terms per batch: their 128-posting work items must fit the item table
    const int items_per_term = T / 128 + 1;
    const int tb = min(kDtThreads, kItemCap / items_per_term);
    // a group whose terms fit one batch keeps their ids, first blocks and entry
    // ranges for all its tiles; only the segment bounds are read per tile
    const bool one_batch = nterm <= tb;
    if (one_batch && (int)threadIdx.x < nterm) {
      const int32_t t = ut[threadIdx.x];
      s_t[threadIdx.x] = t;
      s_tb[threadIdx.x] = (int32_t)__ldg(term_block + t);
      s_e0[threadIdx.x] = __ldg(up + threadIdx.x);
      if ((int)threadIdx.x == nterm - 1) s_e0[nterm] = __ldg(up + nterm);
    }
    int nact = 0;
    if (HEAD) {
      nact = head_nact[g];
      for (int i = threadIdx.x; i < nact; i += blockDim.x) s_hact[i] = __ldg(head_act + (int64_t)g * H + i);
      __syncthreads();
      // FMA head: W[a][q].  Tensor-core head: A fragments of
      // W[q][a] (q < 16 queries, a < nact rows), k-step ks,
      // lane (gid, tig): W[gid][8 ks + tig], W[gid + 8][...], W[gid][8 ks + tig + 4],
      // W[gid + 8][...]; each weight w = high + low, both TF32.  uint8 weights
      // are integers: exact in TF32 and summed exactly in FP32 while every
      // partial sum stays below 2^24 (weights <= 1023, 255 per impact, <= 64 rows)
      if (threadIdx.x == 0) s_tc = HK == kHeadTensor;
      __syncthreads();
      if (HK == kHeadFma)
        for (int i = threadIdx.x; i < nact * kHeadG; i += blockDim.x) {
          const uint32_t raw = __ldg(headw + ((int64_t)g * H + s_hact[i / kHeadG]) * kHeadG + (i % kHeadG));
          memcpy(&s_w[i], &raw, 4);
        }
      if constexpr (HK == kHeadTc05) {
        // B operands W_hi, W_lo [24 rows x 16 queries], K-major without swizzle:
        // row a, query q at float (a / 4) * 64 + q * 4 + a % 4 (core matrices of
        // 8 queries x 4 rows, 128 B); the tensor core reads TF32 (the 13 low
        // mantissa bits ignored), so W_hi = W with those bits cleared and
        // W_lo = W - W_hi carries the rest
        float* whi = reinterpret_cast<float*>(s_af);
        float* wlo = whi + kTc05MaxRows * kHeadG;
        for (int i = threadIdx.x; i < kTc05MaxRows * kHeadG; i += blockDim.x) {
          const int a = i / kHeadG, q = i % kHeadG;
          float w = 0.f;
          if (a < nact) w = __uint_as_float(__ldg(headw + ((int64_t)g * H + s_hact[a]) * kHeadG + q));
          const float hi = __uint_as_float(__float_as_uint(w) & 0xFFFFE000u);
          const int o = (a >> 2) * 64 + q * 4 + (a & 3);
          whi[o] = hi;
          wlo[o] = w - hi;
        }
        tc05::fence_proxy_async_smem();
      }
      const int KS = HK == kHeadTensor ? (nact + 7) / 8 : 0;
      for (int i = threadIdx.x; i < KS * 32; i += blockDim.x) {
        const int ks = i >> 5, gid = (i & 31) >> 2, tig = i & 3;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int q = gid + 8 * (e & 1);
          const int a = 8 * ks + tig + 4 * (e >> 1);
          uint32_t raw = 0u;
          if (a < nact) raw = __ldg(headw + ((int64_t)g * H + s_hact[a]) * kHeadG + q);
          float w;
          if (IMPACT == GS_IMPACT_U8) {
            if ((int32_t)raw > 1023 || (int32_t)raw < 0) s_tc = 0;
            w = (float)(int32_t)raw;
          } else {
            w = __uint_as_float(raw);
          }
          hi[e] = to_tf32(w);
          lo[e] = to_tf32(w - __uint_as_float(hi[e]));
        }
        s_af[2 * i] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        s_af[2 * i + 1] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }

    bool need_clear = true;
    for (int tile_idx = tile_begin; tile_idx < tile_end; ++tile_idx) {
      int tau;
      if (MODE == kModeSample) {
        tau = tile_idx * R;
      } else {
        tau = tile_idx;
        // main pass: a sample tile is scored already; recovery: every tile
        if (MODE == kModeMain && R > 0 && (tau % R) == 0 && tau / R < n_sample) continue;
      }
      const int64_t doc0 = (int64_t)tau * T;
      const int seg_lo = tau * m, seg_hi = min((tau + 1) * m, seg_tiles);
      __syncthreads();  // the previous tile's rows are no longer read
      // the first tile of a unit clears the block; the sample and main
      // epilogues then clear each row as they finish reading it
      if (need_clear || MODE == kModeRecover) {
        uint4* a4 = reinterpret_cast<uint4*>(acc);
        for (int i = threadIdx.x; i < G * T * kCell / 16; i += blockDim.x) a4[i] = make_uint4(0, 0, 0, 0);
        need_clear = false;
      }
      // the planning scan's barriers order the clearing before the tail's
      // reductions; a group without tail terms needs one before the head
      if (nterm == 0) __syncthreads();

      for (int j0 = 0; j0 < nterm; j0 += tb) {
        const int j = j0 + threadIdx.x;
        int items = 0, tiny = 0;
        if (threadIdx.x < tb && j < nterm) {
          const int32_t t = one_batch ? s_t[threadIdx.x] : ut[j];
          const uint32_t* srow = seg + (int64_t)t * (seg_tiles + 1);
          const uint32_t s = __ldg(srow + seg_lo), e = __ldg(srow + seg_hi);
          const int64_t tblk = one_batch ? (int64_t)s_tb[threadIdx.x] : __ldg(term_block + t);
          s_p0[threadIdx.x] = blocks + (tblk + (int64_t)(s >> 5)) * bb;
          s_off[threadIdx.x] = (int32_t)(s & 31u);
          s_len[threadIdx.x] = (int32_t)(e - s);
          if (!one_batch) {
            s_e0[threadIdx.x] = __ldg(up + j);
            if ((int)threadIdx.x == tb - 1 || j == nterm - 1) s_e0[threadIdx.x + 1] = __ldg(up + j + 1);
          }
          if (e - s >= (uint32_t)kTinySeg) items = (int)((((e - 1) >> 5) - (s >> 5)) / 4 + 1);  // chunks of 4 blocks
          else tiny = (int)(e - s);  // short segments are packed 32 postings per warp step
        }
        // one scan of both counts: items (< 2^16 per batch) low, short postings high
        int tot2;
        const int x2 = block_excl_scan(items | (tiny << 16), warp_buf, &tot2);
        const int xi = x2 & 0xffff, xt = x2 >> 16;
        const int total = tot2 & 0xffff, tiny_total = tot2 >> 16;
        if (threadIdx.x < tb) {
          s_item[threadIdx.x] = xi;
          s_tp[threadIdx.x] = xt;
        }
        if (threadIdx.x == 0) s_tp[tb] = tiny_total;
        for (int c = 0; c < items; ++c) item_term[xi + c] = (uint16_t)threadIdx.x;
        // packed chunk c starts inside the short segment that holds posting 32 c
        for (int c = (xt + 31) / 32; 32 * c < xt + tiny; ++c) chunk_j0[c] = (uint16_t)threadIdx.x;
        const int packed = (tiny_total + 31) / 32;
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();
        const int units = total + packed;
        // one (query, weight) entry of the group
        auto entry = [&](int32_t en) {
          uint2 E;
          if (staged) {
            E = ent_s[en - ent_lo];
          } else {
            E = __ldg(ent + en);
            if (scaled) E.y = __float_as_uint(__uint_as_float(E.y) * s_sc[E.x]);
            E.x *= row_bytes;
          }
          return E;
        };
        // one update w x: integer reductions (uint8 impacts, and float impacts
        // in fixed point, w already scaled by 2^S_q), else float reductions
        auto red = [&](auto fxc, uint32_t addr, uint32_t wbits, AccT xv) {
          if constexpr (REC64) {
            const long long v = __float2ll_rn(__uint_as_float(wbits) * (float)xv);
            asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
          } else if constexpr (IMPACT == GS_IMPACT_U8) {
            asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"((int32_t)wbits * (int32_t)xv) : "memory");
          } else if constexpr (decltype(fxc)::value) {
            asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr),
                         "r"(__float2int_rn(__uint_as_float(wbits) * (float)xv))
                         : "memory");
          } else {
            asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(__uint_as_float(wbits) * (float)xv) : "memory");
          }
        };
        // item it: lane l loads posting l of each of its 4 blocks; da = byte
        // offset of the document inside a row, -1 when the lane has no posting
        auto load_item = [&](int it, int* da, AccT* x) -> int {
          const int jj = item_term[it];
          const int c = it - s_item[jj];
          const uint8_t* base = s_p0[jj] + (uint32_t)(4 * c * bb);
          const int rel = 128 * c + lane - s_off[jj];  // segment position of this lane's posting in block 0
          const uint32_t len = (uint32_t)s_len[jj];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            da[i] = lane * kCell;  // no posting: a zero is added to cell `lane` of the row
            x[i] = (AccT)0;
            if ((uint32_t)(rel + 32 * i) < len) {
              const uint8_t* blk = base + i * bb;
              const int32_t doc = __ldg(reinterpret_cast<const int32_t*>(blk) + lane);
              da[i] = (int)(doc - doc0) * kCell;
              if (IMPACT == GS_IMPACT_U8) x[i] = (AccT)__ldg(blk + 128 + lane);
              else x[i] = (AccT)load_x<IMPACT>(blk, lane);
            }
          }
          return jj;
        };
        // NI loaded items of term jj: every entry of the term, every posting
        // (a lane without a posting adds zero to cell `lane`, so the loop
        // needs no predicate)
        auto score_items = [&](auto fxc, auto ni_c, int jj, const int* da, const AccT* x) {
          constexpr int NI = decltype(ni_c)::value;
          const int32_t eb = s_e0[jj], ee = s_e0[jj + 1];
          for (int32_t en = eb; en < ee; ++en) {
            const uint2 E = entry(en);
            const uint32_t row = acc_s + E.x;
#pragma unroll
            for (int i = 0; i < 4 * NI; ++i) red(fxc, row + (uint32_t)da[i], E.y, x[i]);
          }
        };
        // 32 postings of the packed short segments: one posting per lane, its
        // own term and entries
        auto score_packed = [&](auto fxc, int it) {
          const int P = (it - total) * 32 + lane;
          if (P >= tiny_total) return;
          int jj = chunk_j0[it - total];
          while (P >= s_tp[jj + 1]) ++jj;
          const int rel = P - s_tp[jj] + s_off[jj];
          const uint8_t* blk = s_p0[jj] + (uint32_t)((rel >> 5) * bb);
          const int li = rel & 31;
          const int32_t doc = __ldg(reinterpret_cast<const int32_t*>(blk) + li);
          const uint32_t da = (uint32_t)(doc - doc0) * (uint32_t)kCell;
          AccT xv;
          if (IMPACT == GS_IMPACT_U8) xv = (AccT)__ldg(blk + 128 + li);
          else xv = (AccT)load_x<IMPACT>(blk, li);
          const int32_t eb = s_e0[jj], ee = s_e0[jj + 1];
          for (int32_t en = eb; en < ee; ++en) {
            const uint2 E = entry(en);
            red(fxc, acc_s + E.x + da, E.y, xv);
          }
        };
        // units are claimed two at a time; both items' postings are loaded
        // before either is scored, so that each warp keeps 256 postings in
        // flight; the next claim's shared atomic is issued first and read at
        // the end of the iteration, off the loads' critical path
        auto run_units = [&](auto fxc) {
          int nxt_raw = 0;
          if (lane == 0) nxt_raw = atomicAdd(&s_next, 2);
          int nxt = __shfl_sync(0xffffffffu, nxt_raw, 0);
          while (nxt < units) {
            const int it = nxt;
            if (lane == 0) nxt_raw = atomicAdd(&s_next, 2);
            if (it + 1 < total) {
              int da[8];
              AccT x[8];
              const int ja = load_item(it, da, x);
              const int jb = load_item(it + 1, da + 4, x + 4);
              if (ja == jb) {
                score_items(fxc, std::integral_constant<int, 2>{}, ja, da, x);  // consecutive chunks of one segment
              } else {
                score_items(fxc, std::integral_constant<int, 1>{}, ja, da, x);
                score_items(fxc, std::integral_constant<int, 1>{}, jb, da + 4, x + 4);
              }
            } else {
              for (int u = it; u < min(it + 2, units); ++u) {
                if (u < total) {
                  int da[4];
                  AccT x[4];
                  const int jj = load_item(u, da, x);
                  score_items(fxc, std::integral_constant<int, 1>{}, jj, da, x);
                } else {
                  score_packed(fxc, u);
                }
              }
            }
            nxt = __shfl_sync(0xffffffffu, nxt_raw, 0);
          }
        };
        if (fx) run_units(std::true_type{});
        else run_units(std::false_type{});
        __syncthreads();
      }
      if constexpr (REC64) {
        // int64 fixed-point sums -> float rows [G][T], in place: float i
        // takes bytes [4 i, 4 i + 4), inside int64 cell i / 2, so each chunk
        // of cells is read into registers before any of it is written (the
        // writes of a chunk reach only cells of this or earlier chunks)
        constexpr int kPer = 8;
        const long long* a64 = reinterpret_cast<const long long*>(dyn_smem);
        float* af = reinterpret_cast<float*>(dyn_smem);
        const int n_cells = G * T;
        for (int c0 = 0; c0 < n_cells; c0 += kDtThreads * kPer) {
          float v[kPer];
#pragma unroll
          for (int j = 0; j < kPer; ++j) {
            const int i = c0 + j * kDtThreads + (int)threadIdx.x;
            v[j] = i < n_cells && (i >> t_shift) < gq ? __ll2float_rn(a64[i]) * s_isc[i >> t_shift] : 0.f;
          }
          __syncthreads();
#pragma unroll
          for (int j = 0; j < kPer; ++j) {
            const int i = c0 + j * kDtThreads + (int)threadIdx.x;
            if (i < n_cells) af[i] = v[j];
          }
          __syncthreads();
        }
      }

      if (HEAD) {
        // dense head: S[q][d] += sum_a W[q][a] X[a][d] over the group's active
        // head rows a, a contraction of 16 queries x nact rows x T documents.
        const int ib = impact_bytes(IMPACT);
        if constexpr (HK == kHeadTc05) {
          // tensor-memory MMAs (FP32 impacts).  Warpgroup w takes the 128-document
          // M-tiles w, w + 4, ...; thread (warp quarter r, lane l) owns document
          // 32 r + l of the M-tile and tensor-memory lane 32 r + l.  Its head
          // impacts X[a][d] (a < 24) go to columns A_hi (X with the 13 low
          // mantissa bits ignored by the tensor core) and A_lo = X - X_hi; one
          // thread per warpgroup issues D = A_hi W_hi + A_hi W_lo + A_lo W_hi
          // (M = 128 documents, N = 16 queries, K = 8 rows per MMA); every
          // thread then reads its document's 16 query sums and adds them to
          // the tile rows.  The dropped A_lo W_lo term is below 2^-21 of |w x|.
          const int wg = warp >> 2, wq = warp & 3;
          const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
          const uint32_t c_ahi = tmem + (uint32_t)(wg * 64), c_alo = c_ahi + kTc05MaxRows, c_d = c_ahi + 48;
          const int KP = (nact + 7) & ~7;
          constexpr uint32_t kIdesc = tc05::instr_desc(1, 2, 2, 128, 16);
          const float* whi = reinterpret_cast<const float*>(s_af);
          const float* wlo = whi + kTc05MaxRows * kHeadG;
          // the next M-tile's impacts are loaded while the current MMAs run
          uint32_t xs[kTc05MaxRows];
          auto load_x = [&](int mt) {
            const float* xcol = reinterpret_cast<const float*>(head_dense) + doc0 + mt * 128 + wq * 32 + lane;
#pragma unroll
            for (int a = 0; a < kTc05MaxRows; ++a)
              xs[a] = a < nact ? __float_as_uint(__ldg(xcol + (int64_t)s_hact[a] * head_ld)) : 0u;
          };
          const int n_mt = T / 128;
          if (nact > 0 && wg < n_mt) load_x(wg);
          if (nact > 0)
            for (int mt = wg; mt < n_mt; mt += 4) {
              const int dl = mt * 128 + wq * 32 + lane;
#pragma unroll
              for (int c = 0; c < kTc05MaxRows / 8; ++c) {
                if (8 * c >= KP) break;
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  hi[j] = xs[8 * c + j];
                  lo[j] = __float_as_uint(__uint_as_float(hi[j]) - __uint_as_float(hi[j] & 0xFFFFE000u));
                }
                tc05::st_x8(lane_base + c_ahi + 8 * c, hi);
                tc05::st_x8(lane_base + c_alo + 8 * c, lo);
              }
              tc05::wait_st();
              tc05::fence_before();
              wg_barrier(wg);
              if (wq == 0 && lane == 0) {
                tc05::fence_after();
                for (int s8 = 0; s8 < KP / 8; ++s8) {
                  // rows 8 s8 .. 8 s8 + 7: two 16-byte core-matrix columns of B
                  const uint64_t bh = tc05::smem_desc(whi + s8 * 128, 256, 128);
                  const uint64_t bl = tc05::smem_desc(wlo + s8 * 128, 256, 128);
                  tc05::mma_tf32_ts(c_d, c_ahi + 8 * s8, bh, kIdesc, s8 > 0);
                  tc05::mma_tf32_ts(c_d, c_ahi + 8 * s8, bl, kIdesc, 1);
                  tc05::mma_tf32_ts(c_d, c_alo + 8 * s8, bh, kIdesc, 1);
                }
                tc05::commit(&s_mbar[wg]);
              }
              if (mt + 4 < n_mt) load_x(mt + 4);
              // bounded wait; on a timeout every warp still takes the same
              // path (no barrier is left waiting) and the search reports it
              const bool done = tc05::mbar_wait(&s_mbar[wg], mbar_phase, kTc05WaitTries);
              mbar_phase ^= 1u;
              tc_ok = tc_ok && done;
              tc05::fence_after();
              uint32_t dv[16];
              tc05::ld_x16(lane_base + c_d, dv);
              tc05::wait_ld();
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                if (q < gq) {
                  AccT* cell = acc + q * T + dl;
                  *cell = tail_value(*cell, fx, s_isc[q]) + __uint_as_float(dv[q]);
                }
              }
              tc05::fence_before();
            }
          if (fx && nact == 0) {
            // no head rows: fixed-point rows become floats
            for (int i = threadIdx.x; i < gq * T; i += blockDim.x)
              reinterpret_cast<float*>(acc)[i] =
                  tail_value(reinterpret_cast<float*>(acc)[i], true, s_isc[i >> t_shift]);
          }
        } else if (HK == kHeadFma) {
          // CUDA-core FMAs.  Thread (warp w, lane l) owns the 16 queries and
          // documents 2 p, 2 p + 1 of each slab of kSlab documents,
          // p = 32 w + l: the head rows are read coalesced, the next four rows
          // loading while four are multiplied, the weights are warp-wide
          // broadcasts, and every (query, document) cell has one owner (no
          // atomics)
          constexpr int kSlab = 2 * kDtThreads;
          const int dp = warp * 32 + lane;
          for (int slab = 0; slab < T; slab += kSlab) {
            if (slab + 2 * dp >= T) break;  // tiles shorter than one slab
            const int64_t col = doc0 + slab + 2 * dp;
            AccT r[16][2];
#pragma unroll
            for (int i = 0; i < 16; ++i) r[i][0] = r[i][1] = (AccT)0;
            auto load2 = [&](int a, AccT& x0, AccT& x1) {
              const int64_t at = (int64_t)s_hact[a] * head_ld + col;
              if (IMPACT == GS_IMPACT_F32) {
                const float2 u = __ldg(reinterpret_cast<const float2*>(reinterpret_cast<const float*>(head_dense) + at));
                x0 = u.x;
                x1 = u.y;
              } else if (IMPACT == GS_IMPACT_U8) {
                const uint16_t u = __ldg(reinterpret_cast<const uint16_t*>(head_dense + at));
                x0 = (AccT)(u & 0xffu);
                x1 = (AccT)(u >> 8);
              } else {
                const uint32_t u = __ldg(reinterpret_cast<const uint32_t*>(head_dense + at * 2));
                float2 f;
                if (IMPACT == GS_IMPACT_F16) f = __half22float2(*reinterpret_cast<const __half2*>(&u));
                else f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
                x0 = (AccT)f.x;
                x1 = (AccT)f.y;
              }
            };
            // four head rows in registers, the next four already loading
            AccT xn[4][2];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              xn[u][0] = xn[u][1] = (AccT)0;
              if (u < nact) load2(u, xn[u][0], xn[u][1]);
            }
            for (int a0 = 0; a0 < nact; a0 += 4) {
              AccT xs[4][2];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                xs[u][0] = xn[u][0];
                xs[u][1] = xn[u][1];
                xn[u][0] = xn[u][1] = (AccT)0;
                if (a0 + 4 + u < nact) load2(a0 + 4 + u, xn[u][0], xn[u][1]);
              }
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                if (a0 + u >= nact) break;
                const AccT* wr = s_w + (a0 + u) * kHeadG;
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                  AccT w4[4];
                  *reinterpret_cast<uint4*>(w4) = *reinterpret_cast<const uint4*>(wr + 4 * q4);
#pragma unroll
                  for (int v = 0; v < 4; ++v) {
                    if (IMPACT == GS_IMPACT_U8) {
                      r[4 * q4 + v][0] += w4[v] * xs[u][0];
                      r[4 * q4 + v][1] += w4[v] * xs[u][1];
                    } else {
                      r[4 * q4 + v][0] = fmaf((float)w4[v], (float)xs[u][0], (float)r[4 * q4 + v][0]);
                      r[4 * q4 + v][1] = fmaf((float)w4[v], (float)xs[u][1], (float)r[4 * q4 + v][1]);
                    }
                  }
                }
              }
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int q = i;
              if (q < gq) {
                AccT* dst = acc + q * T + slab + 2 * dp;
                uint2 c = *reinterpret_cast<uint2*>(dst);
                AccT* v = reinterpret_cast<AccT*>(&c);
                if constexpr (IMPACT == GS_IMPACT_U8) {
                  v[0] += r[i][0];
                  v[1] += r[i][1];
                } else {
                  v[0] = tail_value(v[0], fx, s_isc[q]) + r[i][0];
                  v[1] = tail_value(v[1], fx, s_isc[q]) + r[i][1];
                }
                *reinterpret_cast<uint2*>(dst) = c;
              }
            }
          }
        } else if (IMPACT != GS_IMPACT_U8 || s_tc) {
          // tensor cores: m16n8k8 TF32 MMAs, M = the 16 queries, K = 8 rows,
          // N = 8 documents.  A warp step covers 8 NT documents base + 0.. as
          // NT MMA tiles: column n of tile j is document base + NT n + j, so
          // that lane (gid, tig) reads documents base + NT gid .. + NT - 1 of a
          // row with one vector load (its B operand for all NT tiles) and owns
          // documents base + 2 NT tig .. + 2 NT - 1 of queries gid, gid + 8 in
          // the D fragments.  Every (query, document) cell has one owner (no
          // atomics).  W = high + low TF32 parts, and X too for FP32 impacts
          // (FP16, BF16 and uint8 impacts are exact in TF32), keeps FP32
          // accuracy; uint8 weights are exact integers: high part only.
          constexpr int NT = 4;
          constexpr int KB = IMPACT == GS_IMPACT_F32 ? 2 : 4;  // k-steps whose operands are loaded together
          using VecT = typename std::conditional<
              IMPACT == GS_IMPACT_U8, uint32_t,
              typename std::conditional<IMPACT == GS_IMPACT_F32, float4, uint2>::type>::type;
          const int gid = lane >> 2, tig = lane & 3;
          const int KS = (nact + 7) / 8;
          for (int cb = warp * 8 * NT; cb < T; cb += kDtThreads / 32 * 8 * NT) {
            const int64_t col = doc0 + cb + NT * gid;
            float d[NT][4];
#pragma unroll
            for (int j = 0; j < NT; ++j) d[j][0] = d[j][1] = d[j][2] = d[j][3] = 0.f;
            for (int k0 = 0; k0 < KS; k0 += KB) {
              VecT xv[KB][2];  // rows 8 ks + tig and 8 ks + tig + 4, NT documents each
#pragma unroll
              for (int u = 0; u < KB; ++u)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int r = 8 * (k0 + u) + tig + 4 * h;
                  xv[u][h] = VecT{};
                  if (r < nact)
                    xv[u][h] = __ldg(reinterpret_cast<const VecT*>(head_dense + ((int64_t)s_hact[r] * head_ld + col) * ib));
                }
#pragma unroll
              for (int u = 0; u < KB; ++u) {
                if (k0 + u >= KS) break;
                const uint4 ah = s_af[2 * ((k0 + u) * 32 + lane)];
                const uint32_t a_hi[4] = {ah.x, ah.y, ah.z, ah.w};
                uint32_t a_lo[4] = {0u, 0u, 0u, 0u};
                if (IMPACT != GS_IMPACT_U8) {
                  const uint4 al = s_af[2 * ((k0 + u) * 32 + lane) + 1];
                  a_lo[0] = al.x; a_lo[1] = al.y; a_lo[2] = al.z; a_lo[3] = al.w;
                }
#pragma unroll
                for (int j = 0; j < NT; ++j) {
                  if constexpr (IMPACT == GS_IMPACT_F32) {
                    // x = high + low TF32 parts as well: three products
                    const float x0 = f4_get(xv[u][0], j), x1 = f4_get(xv[u][1], j);
                    const uint32_t h0 = to_tf32(x0), h1 = to_tf32(x1);
                    const uint32_t l0 = to_tf32(x0 - __uint_as_float(h0)), l1 = to_tf32(x1 - __uint_as_float(h1));
                    mma_tf32(d[j], a_lo, h0, h1);
                    mma_tf32(d[j], a_hi, l0, l1);
                    mma_tf32(d[j], a_hi, h0, h1);
                  } else {
                    const uint32_t b0 = impact_tf32<IMPACT>(xv[u][0], j), b1 = impact_tf32<IMPACT>(xv[u][1], j);
                    if (IMPACT != GS_IMPACT_U8) mma_tf32(d[j], a_lo, b0, b1);
                    mma_tf32(d[j], a_hi, b0, b1);
                  }
                }
              }
            }
            // D: (query gid + 8 h, document cb + 2 NT tig + NT c + j) = d[j][2 h + c]
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int q = gid + 8 * h;
              if (q >= gq) continue;
#pragma unroll
              for (int c = 0; c < 2; ++c) {
                AccT* dst = acc + q * T + cb + 2 * NT * tig + NT * c;
                if constexpr (IMPACT == GS_IMPACT_U8) {
                  int4 v = *reinterpret_cast<int4*>(dst);
                  v.x += __float2int_rn(d[0][2 * h + c]);
                  v.y += __float2int_rn(d[1][2 * h + c]);
                  v.z += __float2int_rn(d[2][2 * h + c]);
                  v.w += __float2int_rn(d[3][2 * h + c]);
                  *reinterpret_cast<int4*>(dst) = v;
                } else {
                  float4 v = *reinterpret_cast<float4*>(dst);
                  const float isc = s_isc[q];
                  v.x = tail_value(v.x, fx, isc) + d[0][2 * h + c];
                  v.y = tail_value(v.y, fx, isc) + d[1][2 * h + c];
                  v.z = tail_value(v.z, fx, isc) + d[2][2 * h + c];
                  v.w = tail_value(v.w, fx, isc) + d[3][2 * h + c];
                  *reinterpret_cast<float4*>(dst) = v;
                }
              }
            }
          }
        } else {
          // uint8 weights too large for exact FP32 sums: integer FMAs, thread
          // (warp w, lane l) owns the 16 queries and documents 2 p, 2 p + 1 of
          // each 1024-document slab, p = 32 w + l
          for (int slab = 0; slab < T; slab += 2 * kDtThreads) {
            const int dp = warp * 32 + lane;
            if (slab + 2 * dp >= T) break;
            const int64_t col = doc0 + slab + 2 * dp;
            int32_t r[16][2];
#pragma unroll
            for (int i = 0; i < 16; ++i) r[i][0] = r[i][1] = 0;
            for (int a = 0; a < nact; ++a) {
              const uint16_t v = __ldg(reinterpret_cast<const uint16_t*>(head_dense + (int64_t)s_hact[a] * head_ld + col));
              const int32_t x0 = v & 0xff, x1 = v >> 8;
              const uint32_t* wr = headw + ((int64_t)g * H + s_hact[a]) * kHeadG;
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const int32_t w = (int32_t)__ldg(wr + i);
                r[i][0] += w * x0;
                r[i][1] += w * x1;
              }
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              if (i < gq) {
                int2* dst = reinterpret_cast<int2*>(acc + i * T + slab + 2 * dp);
                int2 c = *dst;
                c.x += r[i][0];
                c.y += r[i][1];
                *dst = c;
              }
            }
          }
        }
        __syncthreads();
      } else if (fx) {
        // no head: fixed-point rows become floats
        float* af = reinterpret_cast<float*>(acc);
        for (int i = threadIdx.x; i < gq * T; i += blockDim.x) af[i] = tail_value(af[i], true, s_isc[i >> t_shift]);
        __syncthreads();
      }

      // epilogue: each warp step covers 128 documents of one query row (4 per lane)
      const int cpr = T / 128;  // chunks per row
      if (MODE == kModeSample) {
        for (int ci = warp; ci < gq * cpr; ci += kDtThreads / 32) {
          const int ql = ci / cpr;
          const int d0 = (ci - ql * cpr) * 128 + lane * 4;
          *reinterpret_cast<uint4*>(samp + (int64_t)(q0 + ql) * sample_docs + (int64_t)tile_idx * T + d0) =
              *reinterpret_cast<const uint4*>(acc + ql * T + d0);
          *reinterpret_cast<uint4*>(acc + ql * T + d0) = make_uint4(0, 0, 0, 0);
        }
        continue;
      }
      const int64_t n_in = N - doc0;  // documents of this tile inside the collection
      if constexpr (MODE == kModeRecover) {
        if (rec.pass < 3) {
          // radix-select pass: histogram of key digit `pass` (11, 11, 10 bits
          // from the top) over the documents whose higher digits match the
          // prefix resolved so far, warp-aggregated global atomics
          const int shift = rec.pass == 0 ? 21 : (rec.pass == 1 ? 10 : 0);
          const uint32_t pmask = rec.pass == 0 ? 0u : (rec.pass == 1 ? 0xFFE00000u : 0xFFFFFC00u);
          const uint32_t dmask = rec.pass == 2 ? 1023u : 2047u;
          for (int ql = warp; ql < gq; ql += kDtThreads / 32) {
            if (!s_over[ql]) continue;
            const uint32_t pre = s_theta[ql] & pmask;  // pass 0: no digit resolved yet
            const AccT* row = acc + ql * T;
            uint32_t* h = rec.hist + (int64_t)(q0 + ql) * 2048;
            for (int d0 = 0; d0 < T; d0 += 32) {
              const int d = d0 + lane;
              int bin = -1;
              if ((int64_t)d < n_in) {
                const uint32_t key = score_key(row[d]);
                if ((key & pmask) == pre) bin = (int)((key >> shift) & dmask);
              }
              const unsigned peers = __match_any_sync(0xffffffffu, bin);
              if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(h + bin, (uint32_t)__popc(peers));
            }
          }
          continue;
        }
      }
      // candidates above theta_q and the tie bitmap at theta_q.  Each warp owns
      // whole query rows and walks them in windows of 1024 documents: lane l
      // compares documents 128 c + 4 l .. + 3 of chunk c = 0..7 and keeps one bit
      // per document in two masks (above theta_q, equal to theta_q); one warp
      // scan and one global atomic per window reserve the candidate slots, and
      // each lane writes its own candidates.  No block barrier.
      for (int ql = warp; ql < gq; ql += kDtThreads / 32) {
        if (MODE == kModeRecover && !s_over[ql]) continue;  // its top-k is final already
        const int q = q0 + ql;
        const uint32_t th = s_theta[ql];
        const AccT* row = acc + ql * T;
        for (int w0 = 0; w0 < T; w0 += 1024) {
          // one compare per document (score >= theta_q); the few hits are then
          // split into candidates (> theta_q) and ties (== theta_q)
          uint32_t ge_bits = 0;
          const int nc = min(8, (T - w0) / 128);
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if (c >= nc) break;
            const int d0 = w0 + c * 128 + lane * 4;
            const uint4 raw = *reinterpret_cast<const uint4*>(row + d0);
            const uint32_t rv[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              bool ge;
              if (IMPACT == GS_IMPACT_U8) ge = (int32_t)rv[i] >= (int32_t)th;
              else ge = __uint_as_float(rv[i]) >= __uint_as_float(th);
              ge_bits |= (uint32_t)(ge || R <= 0) << (4 * c + i);
            }
          }
          if (n_in < (int64_t)(w0 + 1024)) {
            // the collection ends inside this window: drop documents >= N
            uint32_t keep = 0;
#pragma unroll
            for (int c = 0; c < 8; ++c)
#pragma unroll
              for (int i = 0; i < 4; ++i) keep |= (uint32_t)((int64_t)(w0 + c * 128 + lane * 4 + i) < n_in) << (4 * c + i);
            ge_bits &= keep;
          }
          uint32_t gt_bits = ge_bits, eq_bits = 0;
          if (R > 0) {
            gt_bits = 0;
            for (uint32_t rem = ge_bits; rem; rem &= rem - 1) {
              const int bit = __ffs(rem) - 1;
              const AccT v = row[w0 + (bit >> 2) * 128 + lane * 4 + (bit & 3)];
              bool gt;
              if (IMPACT == GS_IMPACT_U8) gt = (int32_t)v > (int32_t)th;
              else gt = v > __uint_as_float(th);
              if (gt) gt_bits |= 1u << bit;
              else eq_bits |= 1u << bit;
            }
          }
          const int n_gt = __popc(gt_bits);
          int incl = n_gt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          const int tot = __shfl_sync(0xffffffffu, incl, 31);
          if (tot > 0) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&cand_cnt[q], (uint32_t)tot);
            base = __shfl_sync(0xffffffffu, base, 0);
            uint32_t slot = base + (uint32_t)(incl - n_gt);
            while (gt_bits) {
              const int bit = __ffs(gt_bits) - 1;
              gt_bits &= gt_bits - 1;
              const int d = w0 + (bit >> 2) * 128 + lane * 4 + (bit & 3);
              if (slot < cap) cand[(int64_t)q * cap + slot] = make_uint2(score_key(row[d]), (uint32_t)(doc0 + d));
              ++slot;
            }
          }
          if (__any_sync(0xffffffffu, eq_bits != 0)) {
            // tie words: 32 documents = 8 lanes x 4 bits of one chunk
            for (int c = 0; c < nc; ++c) {
              uint32_t word = ((eq_bits >> (4 * c)) & 15u) << (4 * (lane & 7));
              word |= __shfl_xor_sync(0xffffffffu, word, 1);
              word |= __shfl_xor_sync(0xffffffffu, word, 2);
              word |= __shfl_xor_sync(0xffffffffu, word, 4);
              const int64_t wdoc = doc0 + w0 + c * 128 + (lane >> 3) * 32;
              if ((lane & 7) == 0 && word) tiebm[(int64_t)q * bm_words + (wdoc >> 5)] = word;
            }
          }
        }
        if (MODE == kModeMain) {  // the row is read: clear it for the next tile
          __syncwarp();
          for (int d0 = lane * 4; d0 < T; d0 += 128) *reinterpret_cast<uint4*>(acc + ql * T + d0) = make_uint4(0, 0, 0, 0);
        }
      }
    }
  }
  if constexpr (HK == kHeadTc05) {
    if (!tc_ok) {
      // a wait gave up: report it and give the MMAs in flight a last bounded wait
      if ((threadIdx.x & 127) == 0) {
        atomicOr(flags, kFlagTimeout);
        tc05::mbar_wait(&s_mbar[warp >> 2], mbar_phase ^ 1u, kTc05WaitTries);
      }
    }
    tc05::fence_before();
    __syncthreads();
    if (warp == 0) {
      tc05::fence_after();
      tc05::dealloc(tmem, kTc05Cols);
    }
  }
}

// Candidates of the sample tiles (their scores sit in the sample rows).
template <typename ST>
__global__ void dt_sample_emit_kernel(const uint32_t* __restrict__ samp, int64_t sample_docs, int T, int R,
                                      const uint32_t* __restrict__ theta_bits, int k, uint2* __restrict__ cand,
                                      uint32_t* __restrict__ cand_cnt, int64_t cap, uint32_t* __restrict__ tiebm,
                                      int64_t bm_words) {
  const int q = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const uint32_t theta = theta_key<ST>(theta_bits, q, R);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int t_log2 = __ffs(T) - 1;  // T is a power of two
  // uniform per warp: chunks of 32 consecutive sample positions
  for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; i0 < sample_docs; i0 += stride) {
    const int64_t i = i0 + lane;
    const int64_t st = i >> t_log2;  // sample tile st is tile st R
    const int64_t doc = ((st * R) << t_log2) + (i & (int64_t)(T - 1));
    const uint32_t raw = samp[(int64_t)q * sample_docs + i];
    ST v;
    memcpy(&v, &raw, 4);
    const uint32_t key = score_key(v);
    const bool gt = key > theta, tie = key == theta;
    const unsigned mgt = __ballot_sync(0xffffffffu, gt);
    const unsigned mtie = __ballot_sync(0xffffffffu, tie);
    if (lane == 0 && mtie) tiebm[(int64_t)q * bm_words + (doc >> 5)] = mtie;
    if (mgt) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&cand_cnt[q], (uint32_t)__popc(mgt));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (gt) {
        const uint32_t slot = base + (uint32_t)__popc(mgt & ((1u << lane) - 1u));
        if (slot < cap) cand[(int64_t)q * cap + slot] = make_uint2(key, (uint32_t)doc);
      }
    }
  }
}

// Recovery bookkeeping written by the first final pass (device workspace).
struct DtOverflow {
  uint32_t* q_over;   // [B]
  uint32_t* g_mark;   // [ng]
  uint32_t* n_groups;
  int32_t* groups;    // [ng]; NULL: no recovery list (dense rows)
  uint32_t* hist;     // [B][2048]; NULL: nothing to clear
  uint32_t* tiebm;    // [B][bm_words]; NULL: nothing to clear
  int G;
};

// Final exact top-k of each query from its candidates (and ties).
// First pass (REC = false): a query whose candidate list overflowed (more
// documents beat theta_q than the list holds) gets no result here; it is
// marked, its group joins the recovery list, and its histogram row, tie row
// and candidate count are cleared for the recovery passes.  Recovery pass
// (REC = true): only the marked queries, whose candidates now lie above
// their exact k-th score (fewer than k of them) and whose ties sit at it.
template <typename ST, bool REC>
__global__ void __launch_bounds__(1024) dt_final_kernel(const uint2* __restrict__ cand,
                                                        uint32_t* __restrict__ cand_cnt, int64_t cap,
                                                        const uint32_t* __restrict__ tiebm, int64_t bm_words,
                                                        int64_t N, const uint32_t* __restrict__ theta_bits, int R,
                                                        int k, int32_t* __restrict__ out_ids,
                                                        ST* __restrict__ out_scores, uint32_t* flags, DtOverflow ov,
                                                        const int32_t* __restrict__ out_row) {
  __shared__ uint32_t hist[2048];
  __shared__ uint32_t ck[GS_MAX_K];
  __shared__ int32_t cid[GS_MAX_K];
  __shared__ int warp_buf[32];
  __shared__ uint32_t s_digit;
  __shared__ int s_need;
  __shared__ int s_fill;
  const int q = blockIdx.x;
  if (REC && __ldcg(ov.q_over + q) == 0u) return;
  const uint32_t raw = __ldcg(cand_cnt + q);
  if (!REC && raw > cap) {
    if (threadIdx.x == 0) {
      atomicOr(flags, kFlagCandOverflow);
      ov.q_over[q] = 1u;
      cand_cnt[q] = 0u;
      const int g = q / ov.G;
      if (ov.groups && atomicExch(ov.g_mark + g, 1u) == 0u) ov.groups[atomicAdd(ov.n_groups, 1u)] = g;
    }
    if (ov.hist)
      for (int i = threadIdx.x; i < 2048; i += blockDim.x) ov.hist[(int64_t)q * 2048 + i] = 0u;
    if (ov.tiebm)
      for (int64_t w = threadIdx.x; w < bm_words; w += blockDim.x) ov.tiebm[(int64_t)q * bm_words + w] = 0u;
    return;
  }
  const int64_t n = min((int64_t)raw, cap);
  const uint2* c = cand + (int64_t)q * cap;
  if (threadIdx.x == 0) s_fill = 0;
  __syncthreads();
  if (n >= k) {
    select_topk_candidates([&](int64_t i) { return c[i]; }, n, k, hist, warp_buf, &s_digit, &s_need, &s_fill, ck,
                           cid);
  } else {
    // all candidates, then the lowest-id ties at theta_q
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      ck[i] = c[i].x;
      cid[i] = (int32_t)c[i].y;
    }
    const uint32_t theta = theta_key<ST>(theta_bits, q, R);
    const int need_t = k - (int)n;
    int taken = 0;
    const uint32_t* bm = tiebm + (int64_t)q * bm_words;
    for (int64_t w0 = 0; w0 < bm_words && taken < need_t; w0 += blockDim.x) {
      const int64_t w = w0 + threadIdx.x;
      const uint32_t word = w < bm_words ? bm[w] : 0u;
      int tot;
      const int before = taken + block_excl_scan(__popc(word), warp_buf, &tot);
      uint32_t rem = word;
      int r = before;
      while (rem && r < need_t) {
        const int bit = __ffs(rem) - 1;
        rem &= rem - 1;
        const int64_t doc = w * 32 + bit;
        if (doc < N) {
          ck[n + r] = theta;
          cid[n + r] = (int32_t)doc;
        }
        ++r;
      }
      taken += tot;
    }
    __syncthreads();
  }
  int n_pad = 1;
  while (n_pad < k) n_pad <<= 1;
  for (int i = k + threadIdx.x; i < n_pad; i += blockDim.x) {
    ck[i] = 0u;
    cid[i] = 0x7fffffff;
  }
  bitonic_sort_desc(ck, cid, n_pad);
  const int64_t orow = out_row ? (int64_t)__ldg(out_row + q) : (int64_t)q;  // the caller's row of this query
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    out_ids[orow * k + j] = cid[j];
    out_scores[orow * k + j] = key_to_score<ST>(ck[j]);
  }
}

// One radix-select step of the recovery, one CTA per marked query: from the
// histogram of key digit `pass` over the documents that match the prefix
// resolved so far, the digit of the k-th largest key and how many documents
// with the extended prefix still belong to the top k.  The histogram row is
// cleared for the next pass.  After the last digit the prefix is the exact
// k-th largest key, stored as a score (raw bits) in theta.
template <typename ST>
__global__ void __launch_bounds__(1024) dt_over_select_kernel(const uint32_t* __restrict__ q_over,
                                                              uint32_t* __restrict__ hist,
                                                              uint32_t* __restrict__ prefix, int32_t* __restrict__ need,
                                                              uint32_t* __restrict__ theta, int pass, int k) {
  __shared__ uint32_t h[2048];
  __shared__ int warp_buf[32];
  __shared__ uint32_t s_digit;
  __shared__ int s_need;
  const int q = blockIdx.x;
  if (__ldcg(q_over + q) == 0u) return;
  const int nb = pass == 2 ? 1024 : 2048;
  const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
  uint32_t* hr = hist + (int64_t)q * 2048;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    h[i] = __ldcg(hr + i);
    hr[i] = 0u;
  }
  if (threadIdx.x == 0) {
    s_digit = 0u;
    s_need = 1;
  }
  __syncthreads();
  const int need_in = pass == 0 ? k : __ldcg(need + q);
  // thread j sums bins nb - 1 - (j per + u), u < per, counted from the top
  const int per = nb / (int)blockDim.x;
  int local = 0;
  for (int u = 0; u < per; ++u) local += (int)h[nb - 1 - ((int)threadIdx.x * per + u)];
  int tot;
  int above = block_excl_scan(local, warp_buf, &tot);
  for (int u = 0; u < per; ++u) {
    const int b = nb - 1 - ((int)threadIdx.x * per + u);
    const int c = (int)h[b];
    if (above < need_in && need_in <= above + c) {
      s_digit = (uint32_t)b;
      s_need = need_in - above;
    }
    above += c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t pf = (pass == 0 ? 0u : __ldcg(prefix + q)) | (s_digit << shift);
    prefix[q] = pf;
    need[q] = s_need;
    if (pass == 2) {
      const ST v = key_to_score<ST>(pf);
      uint32_t bits;
      memcpy(&bits, &v, 4);
      theta[q] = bits;
    }
  }
}

constexpr size_t kDynSmemFixed = kEntCap * sizeof(uint2) + (kItemCap + kChunkCap) * sizeof(uint16_t);

// Recovery passes keep 8-byte tail accumulators for float impacts.
constexpr size_t rec_acc_bytes(int impact) { return impact == GS_IMPACT_U8 ? kDtMaxAccBytes : 2 * kDtMaxAccBytes; }

// Raises the dynamic shared-memory ceiling of the tile kernels of this form
// and records the recovery kernel's resident CTAs per SM (at its largest
// tile), once per device.  Index builds call it (dt_prepare_device) for every
// head kind of their impact type, so that no search, which a caller may
// capture into a graph, makes the attribute calls.
template <int IMPACT, int HK>
gs_status tile_smem_attr(int* rec_per_sm = nullptr) {
  static std::mutex mu;
  static bool done[128] = {};
  static int rec_ctas[128] = {};
  int dev = 0;
  GS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 128) return GS_ERR_UNSUPPORTED;
  if (!done[dev]) {
    const int ceil_bytes = (int)(kDtMaxAccBytes + kDynSmemFixed);
    const int rec_bytes = (int)(rec_acc_bytes(IMPACT) + kDynSmemFixed);
    GS_CUDA_TRY(cudaFuncSetAttribute(dt_tile_kernel<IMPACT, kModeSample, HK>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, ceil_bytes));
    GS_CUDA_TRY(cudaFuncSetAttribute(dt_tile_kernel<IMPACT, kModeMain, HK>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, ceil_bytes));
    GS_CUDA_TRY(cudaFuncSetAttribute(dt_tile_kernel<IMPACT, kModeRecover, HK>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, rec_bytes));
    int n = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dt_tile_kernel<IMPACT, kModeRecover, HK>,
                                                              kDtThreads, rec_bytes));
    rec_ctas[dev] = std::max(n, 1);
    done[dev] = true;
  }
  if (rec_per_sm) *rec_per_sm = rec_ctas[dev];
  return GS_OK;
}

template <int IMPACT, int HK>
gs_status tile_occupancy(const DtConfig& c, int* ctas) {
  gs_status st = tile_smem_attr<IMPACT, HK>();
  if (st != GS_OK) return st;
  const size_t smem = (size_t)c.G * c.T * 4 + kDynSmemFixed;
  GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, dt_tile_kernel<IMPACT, kModeMain, HK>,
                                                            kDtThreads, smem));
  return GS_OK;
}

template <int IMPACT, int HK>
gs_status launch_tiles_h(const gs_index* ix, const int32_t* q_indptr, int B, int32_t q_nnz, int k, const DtConfig& c,
                         const DtPlan& p, const gs_search_opts* opts, uint32_t* flags, cudaStream_t s) {
  const size_t smem = (size_t)c.G * c.T * 4 + kDynSmemFixed;
  auto ks = dt_tile_kernel<IMPACT, kModeSample, HK>;
  auto km = dt_tile_kernel<IMPACT, kModeMain, HK>;
  gs_status st = tile_smem_attr<IMPACT, HK>();
  if (st != GS_OK) return st;
  // tiles per CTA: enough CTAs for at least 16 waves of resident CTAs
  const int sms = ix->sms > 0 ? ix->sms : 1;
  auto per_cta = [&](int n_tiles) {
    const int64_t items = (int64_t)n_tiles * c.ng;
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, items / (2 * (int64_t)sms * 16)));
  };
  if (c.R > 0) {
    const int ms = per_cta(c.n_sample);
    ks<<<((c.n_sample + ms - 1) / ms) * c.ng, kDtThreads, smem, s>>>(
        ix->blocks, ix->term_block, ix->seg, ix->num_tiles, ix->N, q_indptr, B, q_nnz, c.G, c.T, c.m, c.R, c.ng,
        c.n_sample, p.u_terms, p.u_ptr, p.n_u, p.ent, p.samp, c.sample_docs, p.theta, k, p.cand, p.cand_cnt, c.cap,
        p.tiebm, c.bm_words, ix->head_dense, ix->head_ld, c.H, p.headw, p.head_act, p.head_nact, ms, c.n_sample,
        p.fixp, p.qscale, DtRecover{}, flags);
    GS_LAUNCH_CHECK();
    record_stage(opts, 2, s);
    if (IMPACT == GS_IMPACT_U8)
      kth_score_rows_kernel<int32_t><<<B, kTopkThreads, 0, s>>>(reinterpret_cast<const int32_t*>(p.samp),
                                                               c.sample_docs, c.sample_docs, k, p.theta);
    else
      kth_score_rows_kernel<float><<<B, kTopkThreads, 0, s>>>(reinterpret_cast<const float*>(p.samp), c.sample_docs,
                                                             c.sample_docs, k, p.theta);
    GS_LAUNCH_CHECK();
  } else {
    record_stage(opts, 2, s);
  }
  record_stage(opts, 3, s);
  const int mm = per_cta(c.nt);
  km<<<((c.nt + mm - 1) / mm) * c.ng, kDtThreads, smem, s>>>(
      ix->blocks, ix->term_block, ix->seg, ix->num_tiles, ix->N, q_indptr, B, q_nnz, c.G, c.T, c.m, c.R, c.ng,
      c.n_sample, p.u_terms, p.u_ptr, p.n_u, p.ent, p.samp, c.sample_docs, p.theta, k, p.cand, p.cand_cnt, c.cap,
      p.tiebm, c.bm_words, ix->head_dense, ix->head_ld, c.H, p.headw, p.head_act, p.head_nact, mm, c.nt,
      p.fixp, p.qscale, DtRecover{}, flags);
  GS_LAUNCH_CHECK();
  record_stage(opts, 4, s);
  return GS_OK;
}

// Exact recovery of the queries whose candidate list overflowed (marked by
// the first final pass): a radix select of their exact k-th largest score
// over freshly computed scores of every document (three histogram passes of
// 11, 11 and 10 key bits, each followed by a digit-select kernel), then an
// emission pass of the documents above that score (fewer than k, so the list
// cannot overflow again) and of the ties at it.  Every pass scores each
// document identically (exact integer tail sums), so the four passes agree.
// The grid is persistent: with no marked query every CTA returns at once.
template <int IMPACT, int HK>
gs_status launch_recover_h(const gs_index* ix, const int32_t* q_indptr, int B, int32_t q_nnz, int k,
                           const DtConfig& c, const DtPlan& p, uint32_t* flags, cudaStream_t s) {
  using ST = typename std::conditional<IMPACT == GS_IMPACT_U8, int32_t, float>::type;
  const size_t smem = (size_t)c.G * c.T * (IMPACT == GS_IMPACT_U8 ? 4 : 8) + kDynSmemFixed;
  int per_sm = 1;
  gs_status st = tile_smem_attr<IMPACT, HK>(&per_sm);
  if (st != GS_OK) return st;
  const int sms = ix->sms > 0 ? ix->sms : 1;
  const int tpc = (int)std::max<int64_t>(1, std::min<int64_t>(16, (int64_t)c.nt / (2 * (int64_t)sms)));
  auto kr = dt_tile_kernel<IMPACT, kModeRecover, HK>;
  DtRecover rec{p.ov_groups, p.n_ovg, p.q_over, p.ov_hist, p.ov_prefix, p.ov_theta, 0};
  for (int pass = 0; pass < 4; ++pass) {
    rec.pass = pass;
    kr<<<sms * per_sm, kDtThreads, smem, s>>>(
        ix->blocks, ix->term_block, ix->seg, ix->num_tiles, ix->N, q_indptr, B, q_nnz, c.G, c.T, c.m, c.R, c.ng,
        c.n_sample, p.u_terms, p.u_ptr, p.n_u, p.ent, p.samp, c.sample_docs, p.theta, k, p.cand, p.cand_cnt, c.cap,
        p.tiebm, c.bm_words, ix->head_dense, ix->head_ld, c.H, p.headw, p.head_act, p.head_nact, tpc, c.nt,
        p.fixp, p.qscale, rec, flags);
    GS_LAUNCH_CHECK();
    if (pass < 3) {
      dt_over_select_kernel<ST><<<B, 1024, 0, s>>>(p.q_over, p.ov_hist, p.ov_prefix, p.ov_need, p.ov_theta, pass, k);
      GS_LAUNCH_CHECK();
    }
  }
  return GS_OK;
}

template <int IMPACT>
gs_status launch_tiles(const gs_index* ix, const int32_t* q_indptr, int B, int32_t q_nnz, int k, const DtConfig& c,
                       const DtPlan& p, const gs_search_opts* opts, uint32_t* flags, cudaStream_t s, bool recover) {
  auto go = [&](auto hk) {
    constexpr int HK = decltype(hk)::value;
    if (recover) return launch_recover_h<IMPACT, HK>(ix, q_indptr, B, q_nnz, k, c, p, flags, s);
    return launch_tiles_h<IMPACT, HK>(ix, q_indptr, B, q_nnz, k, c, p, opts, flags, s);
  };
  if (c.HK == kHeadFma) return go(std::integral_constant<int, kHeadFma>{});
  if (c.HK == kHeadTensor) return go(std::integral_constant<int, kHeadTensor>{});
  if (c.HK == kHeadTc05) {
    if constexpr (IMPACT == GS_IMPACT_F32) return go(std::integral_constant<int, kHeadTc05>{});
    return GS_ERR_UNSUPPORTED;
  }
  return go(std::integral_constant<int, kHeadNone>{});
}

// ---- exact top-k of dense score rows ------------------------------------
//
// Rows written densely (the term-parallel and doc-parallel paths) get the same
// sampled-threshold selection as the doc-tiled path: the k-th largest score of
// every R-th chunk of kDenseChunk documents bounds the row's k-th score from
// below; one pass over the row keeps the documents above that bound
// (candidates) and marks those equal to it (ties); the final kernel selects the
// top k of the candidates.  A row whose candidates overflow their list is
// selected again by the radix select over the whole row.

constexpr int kDenseChunk = 1024;

struct DenseConfig {
  int R = 0;  // 0: no sample, the radix select over whole rows
  int n_sample = 0;
  int64_t sample_docs = 0, cap = 0, bm_words = 0;
};

DenseConfig dense_config(const gs_index* ix, int k) {
  DenseConfig c;
  const int nt_full = (int)(ix->N / kDenseChunk);
  int R = kDefaultSampleStride;
  while (R > 1 && (int64_t)((nt_full + R - 1) / R) * kDenseChunk < 2 * (int64_t)k) R /= 2;
  if (R <= 1 || (int64_t)((nt_full + R - 1) / R) * kDenseChunk < (int64_t)k) R = 0;
  c.R = R;
  if (R == 0) return c;
  c.n_sample = (nt_full + R - 1) / R;
  c.sample_docs = (int64_t)c.n_sample * kDenseChunk;
  const int64_t n_round = (ix->N + 255) / 256 * 256;
  c.cap = std::min<int64_t>(n_round, (4 * (int64_t)k * R + 4096 + 255) / 256 * 256);
  c.bm_words = (ix->N + 31) / 32;
  return c;
}

struct DensePlan {
  uint32_t* samp;     // [B][sample_docs]
  uint32_t* theta;    // [B]
  uint2* cand;        // [B][cap]
  uint32_t* cand_cnt; // [B]; cleared block [B cand_cnt][B q_over][B g_mark][n_groups]
  uint32_t* q_over;
  uint32_t* g_mark;
  uint32_t* n_groups;
  uint32_t* tiebm;    // [B][bm_words]
  size_t zero_bytes;
};

DensePlan carve_dense(void* ws, int B, const DenseConfig& c, size_t* bytes) {
  Carver cv(ws);
  DensePlan p{};
  p.samp = cv.take<uint32_t>((size_t)B * std::max<int64_t>(c.sample_docs, 1));
  p.theta = cv.take<uint32_t>(B);
  p.cand = cv.take<uint2>((size_t)B * std::max<int64_t>(c.cap, 1));
  p.zero_bytes = sizeof(uint32_t) * (3 * (size_t)B + 1);
  p.cand_cnt = cv.take<uint32_t>(3 * (size_t)B + 1);
  p.q_over = p.cand_cnt ? p.cand_cnt + B : nullptr;
  p.g_mark = p.cand_cnt ? p.q_over + B : nullptr;
  p.n_groups = p.cand_cnt ? p.g_mark + B : nullptr;
  p.tiebm = cv.take<uint32_t>((size_t)B * std::max<int64_t>(c.bm_words, 1));
  *bytes = cv.size();
  return p;
}

// chunk j R of every row -> sample row (one thread per 16 bytes)
__global__ void dense_sample_gather_kernel(const uint4* __restrict__ rows, int64_t ld4, int R,
                                           uint4* __restrict__ samp, int64_t sample4) {
  const int q = blockIdx.y;
  const int j = blockIdx.x;  // sample chunk
  constexpr int kChunk4 = kDenseChunk / 4;
  for (int i = threadIdx.x; i < kChunk4; i += blockDim.x)
    samp[(int64_t)q * sample4 + (int64_t)j * kChunk4 + i] = rows[(int64_t)q * ld4 + (int64_t)j * R * kChunk4 + i];
}

// One pass over the rows: documents above theta_q become candidates,
// documents equal to it set their bit in the tie bitmap.  A warp takes 4
// consecutive steps of 128 documents (lane l of a step: documents
// 4 l .. 4 l + 3, one 16-byte load), loads all four, and reserves the
// candidate slots of all 512 documents with one atomic: about 0.7% of the
// documents beat theta_q, so most steps hold one and a reservation per step
// would wait on an atomic for most of them.
template <typename ST>
__global__ void __launch_bounds__(256) dense_emit_kernel(const ST* __restrict__ rows, int64_t ld, int64_t N,
                                                         const uint32_t* __restrict__ theta_bits, int R,
                                                         uint2* __restrict__ cand, uint32_t* __restrict__ cand_cnt,
                                                         int64_t cap, uint32_t* __restrict__ tiebm, int64_t bm_words) {
  constexpr int kSteps = 4;
  const int q = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const uint32_t th = theta_key<ST>(theta_bits, q, R);
  const ST* row = rows + (int64_t)q * ld;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t base0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 128 * kSteps; base0 < N;
       base0 += warps * 128 * kSteps) {
    uint32_t key[kSteps][4];
    uint32_t gt[kSteps], eq[kSteps];
#pragma unroll
    for (int u = 0; u < kSteps; ++u) {
      const int64_t d = base0 + 128 * u + 4 * lane;
      // ld is a multiple of 32: the 16 bytes of a document below N lie inside the row
      const uint4 raw = d < N ? __ldcs(reinterpret_cast<const uint4*>(row + d)) : make_uint4(0, 0, 0, 0);
      const uint32_t rv[4] = {raw.x, raw.y, raw.z, raw.w};
      gt[u] = eq[u] = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ST v;
        memcpy(&v, &rv[i], 4);
        key[u][i] = score_key(v);
        const bool in = d + i < N;
        gt[u] |= (uint32_t)(in && key[u][i] > th) << i;
        eq[u] |= (uint32_t)(in && key[u][i] == th) << i;
      }
    }
    const int n = __popc(gt[0]) + __popc(gt[1]) + __popc(gt[2]) + __popc(gt[3]);
    if (__any_sync(0xffffffffu, n != 0)) {
      int incl = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int tot = __shfl_sync(0xffffffffu, incl, 31);
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&cand_cnt[q], (uint32_t)tot);
      base = __shfl_sync(0xffffffffu, base, 0);
      uint32_t slot = base + (uint32_t)(incl - n);
#pragma unroll
      for (int u = 0; u < kSteps; ++u)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if ((gt[u] >> i) & 1u) {
            if (slot < cap)
              cand[(int64_t)q * cap + slot] = make_uint2(key[u][i], (uint32_t)(base0 + 128 * u + 4 * lane + i));
            ++slot;
          }
    }
#pragma unroll
    for (int u = 0; u < kSteps; ++u) {
      if (__any_sync(0xffffffffu, eq[u] != 0)) {
        // tie words: 32 documents = 8 lanes x 4 bits
        uint32_t word = eq[u] << (4 * (lane & 7));
        word |= __shfl_xor_sync(0xffffffffu, word, 1);
        word |= __shfl_xor_sync(0xffffffffu, word, 2);
        word |= __shfl_xor_sync(0xffffffffu, word, 4);
        if ((lane & 7) == 0 && word) tiebm[(int64_t)q * bm_words + (((base0 + 128 * u) >> 5) + (lane >> 3))] = word;
      }
    }
  }
}

}  // namespace

gs_status dense_topk_workspace_bytes(const gs_index* ix, int32_t B, int32_t k, size_t* bytes) {
  const DenseConfig c = dense_config(ix, k);
  if (c.R == 0) {
    *bytes = 0;
    return GS_OK;
  }
  carve_dense(nullptr, B, c, bytes);
  return GS_OK;
}

gs_status dense_topk(const gs_index* ix, const void* rows, int64_t ld, int32_t B, int32_t k, int32_t* out_ids,
                     void* out_scores, void* ws, size_t ws_bytes, uint32_t* flags, cudaStream_t s) {
  const bool is_int = ix->impact == GS_IMPACT_U8;
  const DenseConfig c = dense_config(ix, k);
  if (c.R == 0 || (ld & 31) != 0) {
    if (is_int)
      topk_dense_rows_kernel<int32_t><<<B, kTopkThreads, 0, s>>>(static_cast<const int32_t*>(rows), ld, ix->N, k,
                                                                out_ids, static_cast<int32_t*>(out_scores), nullptr);
    else
      topk_dense_rows_kernel<float><<<B, kTopkThreads, 0, s>>>(static_cast<const float*>(rows), ld, ix->N, k,
                                                              out_ids, static_cast<float*>(out_scores), nullptr);
    GS_LAUNCH_CHECK();
    return GS_OK;
  }
  size_t need = 0;
  DensePlan p = carve_dense(ws, B, c, &need);
  if (need > ws_bytes) return GS_ERR_WORKSPACE;
  GS_CUDA_TRY(cudaMemsetAsync(p.cand_cnt, 0, p.zero_bytes, s));
  GS_CUDA_TRY(cudaMemsetAsync(p.tiebm, 0, sizeof(uint32_t) * (size_t)B * c.bm_words, s));
  dense_sample_gather_kernel<<<dim3((unsigned)c.n_sample, (unsigned)B), 256, 0, s>>>(
      static_cast<const uint4*>(rows), ld / 4, c.R, reinterpret_cast<uint4*>(p.samp), c.sample_docs / 4);
  GS_LAUNCH_CHECK();
  const int sms = ix->sms > 0 ? ix->sms : 1;
  // about 16 resident warps per SM for the whole batch
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ix->N + 4095) / 4096,
                                                                       (int64_t)sms * 16 / std::max(B, 1) + 1));
  const DtOverflow ov{p.q_over, p.g_mark, p.n_groups, nullptr, nullptr, nullptr, 1};
  if (is_int) {
    kth_score_rows_kernel<int32_t><<<B, kTopkThreads, 0, s>>>(reinterpret_cast<const int32_t*>(p.samp), c.sample_docs,
                                                             c.sample_docs, k, p.theta);
    GS_LAUNCH_CHECK();
    dense_emit_kernel<int32_t><<<dim3(gx, (unsigned)B), 256, 0, s>>>(static_cast<const int32_t*>(rows), ld, ix->N,
                                                                     p.theta, c.R, p.cand, p.cand_cnt, c.cap, p.tiebm,
                                                                     c.bm_words);
    GS_LAUNCH_CHECK();
    dt_final_kernel<int32_t, false><<<B, 1024, 0, s>>>(p.cand, p.cand_cnt, c.cap, p.tiebm, c.bm_words, ix->N,
                                                       p.theta, c.R, k, out_ids, static_cast<int32_t*>(out_scores),
                                                       flags, ov, nullptr);
    GS_LAUNCH_CHECK();
    topk_dense_rows_kernel<int32_t><<<B, kTopkThreads, 0, s>>>(static_cast<const int32_t*>(rows), ld, ix->N, k,
                                                              out_ids, static_cast<int32_t*>(out_scores), p.q_over);
  } else {
    kth_score_rows_kernel<float><<<B, kTopkThreads, 0, s>>>(reinterpret_cast<const float*>(p.samp), c.sample_docs,
                                                           c.sample_docs, k, p.theta);
    GS_LAUNCH_CHECK();
    dense_emit_kernel<float><<<dim3(gx, (unsigned)B), 256, 0, s>>>(static_cast<const float*>(rows), ld, ix->N,
                                                                   p.theta, c.R, p.cand, p.cand_cnt, c.cap, p.tiebm,
                                                                   c.bm_words);
    GS_LAUNCH_CHECK();
    dt_final_kernel<float, false><<<B, 1024, 0, s>>>(p.cand, p.cand_cnt, c.cap, p.tiebm, c.bm_words, ix->N, p.theta,
                                                     c.R, k, out_ids, static_cast<float*>(out_scores), flags, ov,
                                                     nullptr);
    GS_LAUNCH_CHECK();
    topk_dense_rows_kernel<float><<<B, kTopkThreads, 0, s>>>(static_cast<const float*>(rows), ld, ix->N, k,
                                                            out_ids, static_cast<float*>(out_scores), p.q_over);
  }
  GS_LAUNCH_CHECK();
  return GS_OK;
}

namespace {

}  // namespace

gs_status dt_prepare_device(const gs_index* ix) {
  const gs_status ost = dt_order_prepare_device();
  if (ost != GS_OK) return ost;
  auto all_heads = [](auto impact_tag) -> gs_status {
    constexpr int I = decltype(impact_tag)::value;
    gs_status st = tile_smem_attr<I, kHeadNone>();
    if (st == GS_OK) st = tile_smem_attr<I, kHeadFma>();
    if (st == GS_OK) st = tile_smem_attr<I, kHeadTensor>();
    if constexpr (I == GS_IMPACT_F32)
      if (st == GS_OK) st = tile_smem_attr<I, kHeadTc05>();
    return st;
  };
  switch (ix->impact) {
    case GS_IMPACT_F32: return all_heads(std::integral_constant<int, GS_IMPACT_F32>{});
    case GS_IMPACT_F16: return all_heads(std::integral_constant<int, GS_IMPACT_F16>{});
    case GS_IMPACT_BF16: return all_heads(std::integral_constant<int, GS_IMPACT_BF16>{});
    default: return all_heads(std::integral_constant<int, GS_IMPACT_U8>{});
  }
}

gs_status dt_plan_info(const gs_index* ix, int32_t B, int32_t k, const gs_search_opts* opts, gs_plan_info* out) {
  DtConfig c;
  gs_status st = dt_config(ix, B, k, opts, &c);
  if (st != GS_OK) return st;
  out->algo = GS_ALGO_DOC_TILED;
  out->group_queries = c.G;
  out->tile_docs = c.T;
  out->sample_stride = c.R;
  out->num_groups = c.ng;
  out->num_tiles = c.nt;
  out->sample_tiles = c.n_sample;
  out->cand_capacity = c.cap;
  out->head_terms = c.H;
  out->query_order = c.order ? 1 : 0;
  int ctas = 0;
  auto occ = [&](auto impact_tag) {
    constexpr int I = decltype(impact_tag)::value;
    if (c.HK == kHeadFma) return tile_occupancy<I, kHeadFma>(c, &ctas);
    if (c.HK == kHeadTensor) return tile_occupancy<I, kHeadTensor>(c, &ctas);
    if (c.HK == kHeadTc05) {
      if constexpr (I == GS_IMPACT_F32) return tile_occupancy<I, kHeadTc05>(c, &ctas);
      return GS_ERR_UNSUPPORTED;
    }
    return tile_occupancy<I, kHeadNone>(c, &ctas);
  };
  switch (ix->impact) {
    case GS_IMPACT_F32: st = occ(std::integral_constant<int, GS_IMPACT_F32>{}); break;
    case GS_IMPACT_F16: st = occ(std::integral_constant<int, GS_IMPACT_F16>{}); break;
    case GS_IMPACT_BF16: st = occ(std::integral_constant<int, GS_IMPACT_BF16>{}); break;
    default: st = occ(std::integral_constant<int, GS_IMPACT_U8>{}); break;
  }
  if (st != GS_OK) return st;
  out->ctas_per_sm = ctas;
  return GS_OK;
}

gs_status dt_order_of(const gs_index* ix, int32_t B, int64_t q_nnz, int32_t k, const gs_search_opts* opts,
                      const void* ws, size_t ws_bytes, int32_t* out_perm, cudaStream_t s) {
  DtConfig c;
  gs_status st = dt_config(ix, B, k, opts, &c);
  if (st != GS_OK) return st;
  if (!c.order) return GS_ERR_UNSUPPORTED;
  size_t need = 0;
  const DtPlan p = carve_dt(const_cast<void*>(ws), ix, B, q_nnz, k, c, &need);
  if (need > ws_bytes) return GS_ERR_WORKSPACE;
  GS_CUDA_TRY(cudaMemcpyAsync(out_perm, p.perm, sizeof(int32_t) * (size_t)B, cudaMemcpyDefault, s));
  return GS_OK;
}

gs_status dt_workspace_bytes(const gs_index* ix, int32_t B, int64_t q_nnz, int32_t k, const gs_search_opts* opts,
                             size_t* bytes) {
  DtConfig c;
  gs_status st = dt_config(ix, B, k, opts, &c);
  if (st != GS_OK) return st;
  carve_dt(nullptr, ix, B, q_nnz, k, c, bytes);
  return GS_OK;
}

gs_status dt_search(const gs_index* ix, const int32_t* q_indptr, const int32_t* q_terms, const float* q_w,
                    int32_t B, int64_t q_nnz, int32_t k, int32_t* out_ids, void* out_scores, void* ws,
                    size_t ws_bytes, uint32_t* flags, const gs_search_opts* opts, cudaStream_t s) {
  DtConfig c;
  gs_status st = dt_config(ix, B, k, opts, &c);
  if (st != GS_OK) return st;
  size_t need = 0;
  DtPlan p = carve_dt(ws, ix, B, q_nnz, k, c, &need);
  if (need > ws_bytes) return GS_ERR_WORKSPACE;
  record_stage(opts, 0, s);
  if (c.order) {
    // the rest of the search runs on the regrouped batch; results go to each query's own row
    st = dt_order(ix, q_indptr, q_terms, q_w, B, (int32_t)q_nnz, c.G, c.H > 0 ? ix->head_slot : nullptr, p.o_indptr,
                  p.o_terms, p.o_w, p.perm, s);
    if (st != GS_OK) return st;
    q_indptr = p.o_indptr;
    q_terms = p.o_terms;
    q_w = p.o_w;
  }
  const int32_t* out_row = c.order ? p.perm : nullptr;
  dt_prep_kernel<<<c.ng, 1024, 0, s>>>(q_indptr, q_terms, q_w, B, (int32_t)q_nnz, c.G, ix->V, ix->impact, p.cnt,
                                       p.u_terms, p.u_ptr, p.n_u, p.ent, ix->head_slot, c.H, p.headw, p.head_act,
                                       p.head_nact, ix->max_abs, p.fixp, p.qscale, flags);
  GS_LAUNCH_CHECK();
  GS_CUDA_TRY(cudaMemsetAsync(p.cand_cnt, 0, p.zero_bytes, s));
  GS_CUDA_TRY(cudaMemsetAsync(p.tiebm, 0, sizeof(uint32_t) * (size_t)B * c.bm_words, s));
  record_stage(opts, 1, s);
  auto tiles = [&](bool recover) {
    switch (ix->impact) {
      case GS_IMPACT_F32:
        return launch_tiles<GS_IMPACT_F32>(ix, q_indptr, B, (int32_t)q_nnz, k, c, p, opts, flags, s, recover);
      case GS_IMPACT_F16:
        return launch_tiles<GS_IMPACT_F16>(ix, q_indptr, B, (int32_t)q_nnz, k, c, p, opts, flags, s, recover);
      case GS_IMPACT_BF16:
        return launch_tiles<GS_IMPACT_BF16>(ix, q_indptr, B, (int32_t)q_nnz, k, c, p, opts, flags, s, recover);
      default:
        return launch_tiles<GS_IMPACT_U8>(ix, q_indptr, B, (int32_t)q_nnz, k, c, p, opts, flags, s, recover);
    }
  };
  st = tiles(false);
  if (st != GS_OK) return st;
  if (c.R > 0) {
    dim3 grid((unsigned)std::min<int64_t>((c.sample_docs + 255) / 256, 64), (unsigned)B);
    if (ix->impact == GS_IMPACT_U8)
      dt_sample_emit_kernel<int32_t><<<grid, 256, 0, s>>>(p.samp, c.sample_docs, c.T, c.R, p.theta, k, p.cand,
                                                          p.cand_cnt, c.cap, p.tiebm, c.bm_words);
    else
      dt_sample_emit_kernel<float><<<grid, 256, 0, s>>>(p.samp, c.sample_docs, c.T, c.R, p.theta, k, p.cand,
                                                        p.cand_cnt, c.cap, p.tiebm, c.bm_words);
    GS_LAUNCH_CHECK();
  }
  const DtOverflow ov{p.q_over, p.g_mark, p.n_ovg, p.ov_groups, p.ov_hist, p.tiebm, c.G};
  if (ix->impact == GS_IMPACT_U8)
    dt_final_kernel<int32_t, false><<<B, 1024, 0, s>>>(p.cand, p.cand_cnt, c.cap, p.tiebm, c.bm_words, ix->N,
                                                       p.theta, c.R, k, out_ids, static_cast<int32_t*>(out_scores),
                                                       flags, ov, out_row);
  else
    dt_final_kernel<float, false><<<B, 1024, 0, s>>>(p.cand, p.cand_cnt, c.cap, p.tiebm, c.bm_words, ix->N, p.theta,
                                                     c.R, k, out_ids, static_cast<float*>(out_scores), flags, ov,
                                                     out_row);
  GS_LAUNCH_CHECK();
  // Without a sample every document is a candidate (cap >= N): no list can
  // overflow.  With one, the queries the first final pass marked are
  // recomputed exactly; with none marked these launches return at once.
  if (c.R > 0) {
    st = tiles(true);
    if (st != GS_OK) return st;
    if (ix->impact == GS_IMPACT_U8)
      dt_final_kernel<int32_t, true><<<B, 1024, 0, s>>>(p.cand, p.cand_cnt, c.cap, p.tiebm, c.bm_words, ix->N,
                                                        p.ov_theta, 1, k, out_ids,
                                                        static_cast<int32_t*>(out_scores), flags, ov, out_row);
    else
      dt_final_kernel<float, true><<<B, 1024, 0, s>>>(p.cand, p.cand_cnt, c.cap, p.tiebm, c.bm_words, ix->N,
                                                      p.ov_theta, 1, k, out_ids, static_cast<float*>(out_scores),
                                                      flags, ov, out_row);
    GS_LAUNCH_CHECK();
  }
  record_stage(opts, 5, s);
  return GS_OK;
}

}  // namespace gs
