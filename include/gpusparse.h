/*
 * gpusparse.h -- exact batched sparse scoring on a GPU-resident inverted index
 * (GB300, sm_103a).  C ABI: plain pointers and sizes, no framework types.
 *
 * Problem (Sec. 4.1, Eq. 4-5 of "GPUSparse: GPU-Accelerated Learned Sparse
 * Retrieval with Parallel Inverted Indices"): for each query q = {(t_i, w_i)}
 * of a batch and every document d of the collection,
 *     score(q, d) = sum_i w_i * s_d(t_i),
 * with s_d(t) the impact the index stores for (d, t) (0 if absent), computed
 * by scatter-adding every posting of every query term (no pruning, Sec. 4.3);
 * then the exact top-k of each query under the order (score descending,
 * document id ascending).  All N documents are eligible, including those that
 * score 0.
 *
 * Index layout (Sec. 3.2, Eq. 2-3): term-major posting lists, each sorted by
 * document id and padded to a multiple of W = 32 postings with (doc -1,
 * impact 0).  Every 32-posting block is stored contiguously as
 * [32 x int32 doc ids][32 x impact], so both halves are 128-bit loadable.
 *
 * Conventions for every entry point:
 *   - "device" pointers must point to memory of the current CUDA device;
 *     "host" pointers to host memory (pinned for the copies to overlap).
 *   - stream: a cudaStream_t (NULL = the legacy default stream).  Calls are
 *     asynchronous on it unless stated; inputs must stay valid until the work
 *     enqueued on the stream has run.
 *   - the caller owns every input, output and workspace buffer; the library
 *     owns gs_index objects and never allocates inside gs_search.
 *   - argument errors are reported synchronously by the return value; data
 *     errors found on the device (a query term id outside [0, V), a
 *     non-finite query weight) skip the offending query term and set a flag
 *     word in the workspace, read with gs_search_flags().
 *   - no entry point is thread-safe against a concurrent gs_index_free of the
 *     same index.
 */
#ifndef GPUSPARSE_H
#define GPUSPARSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* gs_stream_t; /* identical to cudaStream_t */

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1,   /* null pointer, bad size, k > N, ... */
  GS_ERR_OUT_OF_MEMORY = 2, /* index build could not allocate */
  GS_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  GS_ERR_UNSUPPORTED = 4,   /* valid but not supported (k > GS_MAX_K, ...) */
  GS_ERR_DATA = 5,          /* invalid document data at index build; from a
                               synchronous search call: the device skipped
                               invalid query data (GS_FLAG_BAD_*) */
  GS_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
  GS_ERR_WORKSPACE = 7      /* workspace smaller than gs_search_workspace_size() */
} gs_status;

/* Stored impact type of the index (the paper stores float32, Sec. 3.2;
 * reduced precisions follow its future-work item 2, Sec. 8).
 *   F32  : float32 impacts, float32 accumulation, float32 scores.
 *   F16  : IEEE binary16 impacts (nearest-even), float32 accumulation.
 *   BF16 : bfloat16 impacts (nearest-even), float32 accumulation.
 *   U8   : uint8 impacts round(w * 255 / 5) (nearest-even of 51 w, document
 *          weights must lie in [0, 5]); query weights are quantised by the
 *          same rule, clamped to [0, 255]; int32 accumulation and int32 scores
 *          (exact: a query may hold at most GS_MAX_QUERY_TERMS_U8 terms). */
typedef enum { GS_IMPACT_F32 = 0, GS_IMPACT_F16 = 1, GS_IMPACT_BF16 = 2, GS_IMPACT_U8 = 3 } gs_impact;

/* Scoring kernels.
 *   TERM_PARALLEL : the paper's batched scatter-add (Sec. 4.2, 5.2): every
 *                   (query, term, posting chunk) work item adds its
 *                   contributions into dense [B x N] score rows with global
 *                   atomics; then a radix-select top-k over the rows.
 *   DOC_TILED     : a doc tile of the score rows of a group of queries lives
 *                   in shared memory; every (term, tile) posting segment is
 *                   read once per group (the hybrid kernel of Sec. 8, future
 *                   work 1).  Candidates above a per-query threshold taken
 *                   from a sampled subset of tiles are kept; the dense rows
 *                   are never written.
 *   DOC_PARALLEL  : one thread per (query, document): walks the document's
 *                   terms against a dense query vector (Sec. 5.3), no atomics.
 *   AUTO          : DOC_TILED when the index has a tile table, else
 *                   TERM_PARALLEL. */
typedef enum {
  GS_ALGO_AUTO = 0,
  GS_ALGO_TERM_PARALLEL = 1,
  GS_ALGO_DOC_TILED = 2,
  GS_ALGO_DOC_PARALLEL = 3
} gs_algo;

#define GS_BLOCK 32                  /* W, postings per block (Sec. 3.2, Eq. 2) */
#define GS_MAX_K 2048                /* largest supported k */
#define GS_MAX_QUERY_TERMS_U8 33000  /* 255 * 255 * 33000 < 2^31 */

/* flag bits of the workspace flag word */
#define GS_FLAG_BAD_TERM 1u     /* a query term id outside [0, V) was skipped */
#define GS_FLAG_BAD_WEIGHT 2u   /* a non-finite query weight was skipped */
#define GS_FLAG_CAND_OVERFLOW 4u/* doc-tiled, informational: more documents beat
                                   a query's sampled threshold than its
                                   candidate list holds; that query's top-k
                                   was recomputed exactly (radix select of
                                   its k-th score over fresh scores of every
                                   document), so the results stay exact */
#define GS_FLAG_TIMEOUT 8u      /* a bounded device wait gave up (the
                                   tensor-memory head waiting for its MMAs):
                                   results of that call are undefined */
#define GS_FLAG_BAD_INDPTR 16u  /* the query CSR row pointer was not monotone
                                   or ended past q_nnz: results undefined */

typedef struct gs_index gs_index;

#define GS_MAX_HEAD_TERMS 64

typedef struct {
  int32_t tile_docs;  /* documents per tile of the segment table used by the
                         doc-tiled kernel: a power of two in [256, 65536];
                         0 = default (1024); -1 = build no table */
  int32_t head_terms; /* dense head: the H terms with the longest posting
                         lists also get a dense [H x N] impact matrix that the
                         doc-tiled kernel multiplies (FMAs or tensor-core
                         MMAs) instead of scattering them; 0 = default (24
                         for FP32 impacts, 64 otherwise), -1 = none, at most
                         GS_MAX_HEAD_TERMS */
  int32_t doc_major;  /* 1: also keep a document-major copy (doc CSR of stored
                         impacts) for the DOC_PARALLEL kernel */
  int32_t reserved[5];
} gs_build_opts;

typedef struct {
  int64_t num_docs;
  int64_t postings;         /* non-zeros of the collection */
  int64_t padded_postings;  /* sum of padded_length(t) (Sec. 3.2, Eq. 2) */
  int64_t blocks;           /* padded_postings / 32 */
  int64_t posting_bytes;    /* blocks * block_bytes */
  int64_t meta_bytes;       /* per-term arrays and the tile segment table */
  int32_t vocab;
  int32_t impact;           /* gs_impact */
  int32_t block_bytes;      /* 256 (F32), 192 (F16/BF16), 160 (U8) */
  int32_t tile_docs;        /* 0 when no tile table was built */
  int32_t num_tiles;
  int32_t score_is_int;     /* 1 on the U8 path: scores are int32 */
  int32_t head_terms;       /* H of the dense head (0: none) */
  int32_t reserved0;
  int64_t head_bytes;       /* bytes of the dense head matrix */
} gs_index_stats;

/* Read-only views of the index's device arrays (for inspection and tests).
 * block b of term t is b in [term_block[t], term_block[t + 1]).  seg is
 * [vocab][num_tiles + 1]: seg[t * (num_tiles + 1) + j] is the position
 * within the list of t of its first posting with doc id >= j * tile_docs. */
typedef struct {
  const void* blocks;         /* blocks * block_bytes bytes */
  const int64_t* term_block;  /* [vocab + 1] */
  const int32_t* term_len;    /* [vocab] postings of each list, unpadded */
  const float* max_score;     /* [vocab] largest stored impact of each list */
  const uint32_t* seg;        /* see above; NULL without a tile table */
  const int32_t* head_term;   /* [head_terms] term ids of the dense head */
  const void* head_dense;     /* [head_terms][head_ld] impacts (index type) */
  int64_t head_ld;            /* row length of head_dense, >= num_docs */
  const int64_t* doc_indptr;  /* document-major copy (NULL unless built) */
  const int32_t* doc_terms;
  const void* doc_impacts;    /* stored impacts, index type */
} gs_index_layout;

/* Stage boundaries at which gs_search records the caller's CUDA events when
 * gs_search_opts.stage_events is set (timing only; no work is skipped):
 *   [0] start  [1] after query prep  [2] after sample scoring (DOC_TILED) or
 *   score-row zeroing (TERM_PARALLEL)  [3] after the sample top-k
 *   [4] after the main scoring kernel  [5] end, after the final top-k. */
#define GS_NUM_STAGE_EVENTS 6

typedef struct {
  int32_t algo;          /* gs_algo */
  int32_t group_queries; /* DOC_TILED: queries per group (0 = auto) */
  int32_t tile_docs;     /* DOC_TILED: docs per tile, a multiple of the
                            index's tile_docs (0 = auto) */
  int32_t chunk_blocks;  /* TERM_PARALLEL: blocks per work item (0 = auto) */
  int32_t sample_stride; /* DOC_TILED: 1 of every R tiles forms the threshold
                            sample (0 = auto, 1 = no sampling: every
                            document is a candidate) */
  int32_t use_head;      /* DOC_TILED dense head (requires 16 queries per
                            group and an index with a head): 0 = auto
                            (FMAs for FP32 impacts, warp-level tensor-core
                            MMAs otherwise),
                            1 = CUDA-core FMAs, 2 = warp-level tensor-core
                            MMAs (mma.sync), 3 = tensor-memory MMAs (tcgen05,
                            FP32 impacts and heads of at most 24 rows only,
                            else GS_ERR_UNSUPPORTED), -1 = off */
  void* const* stage_events; /* NULL, or GS_NUM_STAGE_EVENTS cudaEvent_t */
  int32_t query_order;   /* DOC_TILED, groups of 8 queries or more: 1 =
                            regroup the batch (two groups or more) so that
                            queries sharing long sparse-tail posting lists
                            share a group (each tile segment of a shared term
                            is then read once for all of them; results are
                            written at each query's own row and are the same
                            as in the caller's order); 0 = regroup only where
                            the library's cost model predicts a gain (at least
                            4 groups and batch x documents large enough:
                            about 64 queries over 8.8M documents on GB300);
                            -1 = keep the caller's order */
} gs_search_opts;

/* --- index --------------------------------------------------------------- */

/* Builds the index (Sec. 3.2) from documents given as CSR on the device:
 *   doc_indptr [num_docs + 1] int64, doc_indptr[0] = 0, non-decreasing,
 *               doc_indptr[num_docs] = nnz;
 *   doc_terms  [nnz] int32 term ids in [0, vocab), no term twice in a doc;
 *   doc_w      [nnz] float32 finite weights (U8: in [0, 5]; F16: within the
 *               binary16 range).
 * Runs on `stream` and synchronises it before returning.  Returns
 * GS_ERR_DATA for invalid document data (no index is created),
 * GS_ERR_OUT_OF_MEMORY when device memory runs out.  *out receives a
 * library-owned handle, released with gs_index_free. */
gs_status gs_index_build(const int64_t* doc_indptr, const int32_t* doc_terms, const float* doc_w,
                         int64_t num_docs, int64_t nnz, int32_t vocab, gs_impact impact,
                         gs_stream_t stream, gs_index** out);

/* Same with build options (NULL = defaults). */
gs_status gs_index_build_ex(const int64_t* doc_indptr, const int32_t* doc_terms, const float* doc_w,
                            int64_t num_docs, int64_t nnz, int32_t vocab, gs_impact impact,
                            const gs_build_opts* opts, gs_stream_t stream, gs_index** out);

/* Sizes of the index (the block layout of Sec. 3.2, Eq. 2, and the memory
 * accounting of Sec. 3.3: posting bytes = padded postings x (4 + impact
 * bytes)).  Host call, no device work. */
gs_status gs_index_info(const gs_index* index, gs_index_stats* out);
/* Device addresses of the index arrays of Sec. 3.2 (see gs_index_layout);
 * the views stay valid until gs_index_free. */
gs_status gs_index_get_layout(const gs_index* index, gs_index_layout* out);
/* Releases the index and all its device memory (Sec. 3.3's footprint);
 * NULL is ignored.  No search on it may be in flight. */
void gs_index_free(gs_index* index);

/* --- search -------------------------------------------------------------- */

/* Device workspace bytes gs_search / gs_score_dense need for a batch of
 * `batch` queries holding `q_nnz` terms in total, with top-`k` (k is
 * ignored by gs_score_dense).  opts may be NULL.  host_io != 0 adds room
 * for gs_search_host's device copies of the queries and results.  This is
 * the score-buffer memory of Sec. 7 (limitation 3): B x N score rows on the
 * term-parallel path, per-query candidate lists and tie bitmaps on the
 * doc-tiled path. */
gs_status gs_search_workspace_size(const gs_index* index, int32_t batch, int64_t q_nnz, int32_t k,
                                   const gs_search_opts* opts, int32_t host_io, size_t* bytes);

/* Exact top-k of a batch of queries (Sec. 4, Eq. 4-5 + exact top-k).
 * Queries are CSR on the device:
 *   q_indptr [batch + 1] int32, q_indptr[0] = 0, non-decreasing,
 *             q_indptr[batch] <= q_nnz;
 *   q_terms  [q_nnz] int32 term ids; q_w [q_nnz] float32 weights.
 *   q_nnz is the capacity of q_terms / q_w: entries past q_indptr[batch]
 *   are ignored (a captured graph can serve batches of fewer terms).
 *   A term may repeat inside a query: every occurrence contributes.
 * Outputs on the device, row-major [batch x k]:
 *   out_ids    int32 document ids, ordered by (score desc, id asc);
 *   out_scores float32 scores (int32 on the U8 path).
 * Scores are those of Eq. 4 over the stored impacts: exact on the U8 path;
 * on float paths within 1e-5 * sum |w x| + 1e-6 of the exact value, the
 * order taken by the returned scores.
 * 1 <= k <= min(N, GS_MAX_K).  workspace: device, >= the size reported by
 * gs_search_workspace_size for the same arguments, 256-byte aligned; it is
 * used as scratch and must not be shared by calls that overlap on the GPU.
 * Asynchronous on `stream`; never synchronises or allocates. */
gs_status gs_search(const gs_index* index, const int32_t* q_indptr, const int32_t* q_terms,
                    const float* q_w, int32_t batch, int64_t q_nnz, int32_t k, int32_t* out_ids,
                    void* out_scores, void* workspace, size_t workspace_bytes,
                    const gs_search_opts* opts, gs_stream_t stream);

/* gs_search with the queries and results in host memory: copies the queries
 * to the workspace, searches, copies the results back and synchronises the
 * stream before returning.  The workspace must be sized with host_io = 1.
 * Returns GS_ERR_DATA when the device skipped invalid query data (a flag of
 * GS_FLAG_BAD_TERM, _BAD_WEIGHT or _BAD_INDPTR; gs_search_flags on the same
 * workspace tells which); the results are written all the same, computed
 * without the skipped terms. */
gs_status gs_search_host(const gs_index* index, const int32_t* h_q_indptr, const int32_t* h_q_terms,
                         const float* h_q_w, int32_t batch, int64_t q_nnz, int32_t k,
                         int32_t* h_out_ids, void* h_out_scores, void* workspace,
                         size_t workspace_bytes, const gs_search_opts* opts, gs_stream_t stream);

/* The dense score rows of Eq. 4 without top-k: out_rows [batch x num_docs]
 * on the device, float32 (int32 on the U8 path).  Same query and workspace
 * conventions as gs_search; the term-parallel scatter-add computes them. */
gs_status gs_score_dense(const gs_index* index, const int32_t* q_indptr, const int32_t* q_terms,
                         const float* q_w, int32_t batch, int64_t q_nnz, void* out_rows,
                         void* workspace, size_t workspace_bytes, gs_stream_t stream);

/* The plan gs_search resolves for these arguments (kernel, tile shapes,
 * sample stride), for inspection and performance accounting. */
typedef struct {
  int32_t algo;          /* resolved gs_algo */
  int32_t group_queries; /* DOC_TILED: G */
  int32_t tile_docs;     /* DOC_TILED: T */
  int32_t sample_stride; /* DOC_TILED: R (0: no sample, every doc a candidate) */
  int32_t num_groups;
  int32_t num_tiles;
  int32_t sample_tiles;  /* tiles j * R, j < sample_tiles, form the sample */
  int32_t chunk_blocks;  /* TERM_PARALLEL: blocks per work item */
  int64_t cand_capacity; /* DOC_TILED: candidate slots per query */
  int32_t head_terms;    /* DOC_TILED: dense head terms used (0: none) */
  int32_t ctas_per_sm;   /* DOC_TILED: resident CTAs per SM of the scoring
                            kernel (occupancy calculator) */
  int64_t query_order;   /* DOC_TILED: 1 = the batch is regrouped by shared
                            tail terms (gs_search_opts.query_order) */
  int64_t reserved[2];
} gs_plan_info;

gs_status gs_search_plan(const gs_index* index, int32_t batch, int64_t q_nnz, int32_t k,
                         const gs_search_opts* opts, gs_plan_info* out);

/* The query groups of the last DOC_TILED gs_search that used `workspace` with
 * the same index, batch, q_nnz, k and opts, when that search regrouped the
 * batch (gs_plan_info.query_order = 1): writes out_perm[p] = the caller's
 * query at position p of the regrouped batch, whose group g holds positions
 * [g G, g G + G) (G = gs_plan_info.group_queries).  For performance accounting
 * (the tiles' postings are read once per group and distinct term, Sec. 4.1,
 * Sec. 8 future work 1).  out_perm: [batch] int32, device or page-locked host
 * memory; the copy is asynchronous on `stream`, after the search.  Returns
 * GS_ERR_UNSUPPORTED when these arguments do not regroup (another algorithm,
 * groups of fewer than 8 queries, a single group, query_order = -1). */
gs_status gs_search_query_order(const gs_index* index, int32_t batch, int64_t q_nnz, int32_t k,
                                const gs_search_opts* opts, const void* workspace, size_t workspace_bytes,
                                int32_t* out_perm, gs_stream_t stream);

/* Merge of per-shard top-k lists (documents sharded across GPUs or across
 * indexes: each shard holds a contiguous range of document ids and returns
 * local ids).  shard_ids[s] / shard_scores[s] point to [batch x k_in] device
 * arrays of shard s, ordered as gs_search returns them; doc_offset[s] (host)
 * is added to its ids.  Writes the global top-k (k <= n_shards * k_in,
 * k <= GS_MAX_K) by (score desc, id asc) to out_ids / out_scores [batch x k]
 * on the device.  Scores are float32, or int32 when score_is_int != 0.
 * n_shards <= GS_MAX_SHARDS.  Asynchronous on `stream`. */
#define GS_MAX_SHARDS 64
gs_status gs_merge_topk(const int32_t* const* shard_ids, const void* const* shard_scores,
                        const int64_t* doc_offset, int32_t n_shards, int32_t batch, int32_t k_in, int32_t k,
                        int32_t score_is_int, int32_t* out_ids, void* out_scores, gs_stream_t stream);

/* Synchronises `stream`, then returns in *flags the GS_FLAG_* bits the last
 * call that used `workspace` raised (the flag word leads the workspace; the
 * data-error flags are those of the query checks of Sec. 4.2's batching step,
 * the overflow flag that of the candidate lists). */
gs_status gs_search_flags(const void* workspace, gs_stream_t stream, uint32_t* flags);

/* --- uneven batches from captured CUDA graphs -----------------------------
 *
 * A runner owns device buffers for up to max_batch queries / max_q_nnz query
 * terms / max_k results, a workspace and one CUDA graph per (batch bucket, k):
 * batches are padded to a power-of-two bucket with empty queries.  The first
 * batch of a bucket is used to time candidate doc-tiled plans (tile length,
 * queries per group, sample stride, dense head; autotune != 0) — the
 * grid-search analogue of the paper's BLOCK_PL tuning (Sec. 5.2) — and the
 * chosen plan's gs_search is captured into a graph that later batches replay
 * with one launch.  Queries and results are in host memory; the work runs
 * on the runner's own stream after the work already queued on `stream`, and
 * the call returns when the results are in host memory.  gs_runner_create allocates (device and pinned host
 * memory); gs_runner_search does not.  A runner serialises its own calls. */
typedef struct gs_runner gs_runner;

gs_status gs_runner_create(const gs_index* index, int32_t max_batch, int64_t max_q_nnz, int32_t max_k,
                           const gs_search_opts* opts, int32_t autotune, gs_runner** out);
/* Returns GS_ERR_DATA, with the results written, when the device skipped
 * invalid query data (as gs_search_host does). */
gs_status gs_runner_search(gs_runner* runner, const int32_t* h_q_indptr, const int32_t* h_q_terms,
                           const float* h_q_w, int32_t batch, int32_t k, int32_t* h_out_ids,
                           void* h_out_scores, gs_stream_t stream);
/* the plan a bucket runs with (after its first batch), and its tuned time */
gs_status gs_runner_plan(gs_runner* runner, int32_t batch, int32_t k, gs_search_opts* out_opts,
                         float* out_tuned_ms);
void gs_runner_free(gs_runner* runner);

/* --- serving loop with continuous batching --------------------------------
 *
 * (Sec. 8, future work 3: streaming query batching.)  Requests — one query,
 * its k, the index it targets — are submitted from any host thread and
 * queued.  A lane is one admission slot: a stream, a search workspace (the
 * score memory of one batch), device and pinned buffers; the number of lanes
 * follows from workspace_budget_bytes (when > 0) and `lanes`, so requests are
 * admitted as score-buffer memory frees up.  A scheduler thread forms a batch
 * from the oldest pending request's index whenever a lane is free (optionally
 * waiting up to max_wait_us for more requests) and runs it on the lane's
 * stream; batches of different lanes overlap on the GPU.  Each lane's
 * completion thread hands every request the first k results of its batch
 * (the batch runs with the largest k among its requests).  Several indexes
 * may be resident at once.  Waits are bounded: gs_server_wait returns
 * GS_ERR_TIMEOUT after timeout_us and the request can be waited for again. */
typedef struct gs_server gs_server;

typedef struct {
  int32_t lanes;                  /* admission slots (batches in flight) */
  int32_t max_batch;              /* queries per batch */
  int32_t max_q_nnz;              /* query terms per batch */
  int32_t max_k;                  /* largest k a request may ask for */
  int32_t max_wait_us;            /* accumulation window once a lane is free (0 = none) */
  int32_t reserved;
  int64_t workspace_budget_bytes; /* > 0: lanes = min(lanes, budget / lane workspace) */
  gs_search_opts opts;            /* search plan for every batch */
} gs_server_config;

typedef struct {
  int32_t lanes;
  int32_t max_in_flight;          /* most lanes busy at once */
  int64_t completed;
  int64_t batches;
  int64_t batched_queries;        /* sum of batch sizes */
  int64_t queued;                 /* requests waiting for a lane */
  int64_t lane_workspace_bytes;
} gs_server_stats;

/* indexes: n_indexes resident indexes (owned by the caller, kept alive until
 * gs_server_destroy); index ids in requests are positions in this array. */
gs_status gs_server_create(const gs_index* const* indexes, int32_t n_indexes, const gs_server_config* cfg,
                           gs_server** out);
/* copies the query (host memory); *ticket identifies the request.  A term id
 * outside [0, V) of the target index or a non-finite weight is rejected here
 * with GS_ERR_INVALID_ARG. */
gs_status gs_server_submit(gs_server* server, int32_t index_id, const int32_t* terms, const float* weights,
                           int32_t nnz, int32_t k, int64_t* ticket);
/* waits at most timeout_us for the request; on GS_OK writes k ids and k
 * scores (float32, int32 on uint8 indexes) to host memory and, when
 * latency_us is not NULL, the time from submit to completion.  A batch whose
 * search failed, or raised a data-error flag, gives each of its requests that
 * status (GS_ERR_CUDA, GS_ERR_DATA). */
gs_status gs_server_wait(gs_server* server, int64_t ticket, int32_t* out_ids, void* out_scores, int64_t timeout_us,
                         double* latency_us);
gs_status gs_server_stats_get(gs_server* server, gs_server_stats* out);
/* stops the threads after the batches in flight complete; queued requests are dropped */
void gs_server_destroy(gs_server* server);

/* --- search without allocation (the paper has no counterpart) ------------
 *
 * Some callers cannot call cudaMalloc: code that runs where another
 * allocator owns all of the device's memory (a host framework's fixed pool,
 * a memory-capped sandbox), and latency-critical request paths where
 * cudaMalloc / cudaFree would synchronise the device.  gs_search_static
 * serves them: it is gs_search with its scratch taken from one file-scope
 * array of device memory of GS_STATIC_SCRATCH_BYTES that every GPU which
 * loads the library holds until the process exits.  The caller still
 * passes the queries and the output arrays (device memory, as for
 * gs_search).
 *   - Batches whose workspace (gs_search_workspace_size) exceeds
 *     GS_STATIC_SCRATCH_BYTES are rejected with GS_ERR_WORKSPACE; nothing is
 *     allocated then either.
 *   - The first call on a device looks the array's device address up with
 *     cudaGetSymbolAddress (with that device current); make that first call
 *     before any stream capture.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; the search clears what it needs itself.  Calls that overlap on
 *     the GPU (other streams, other host threads) race on the array: serialise
 *     them.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine.
 *   - Its flag word is read with gs_search_static_flags() (gs_search_flags()
 *     takes a workspace pointer); data errors skip the offending query terms
 *     as in gs_search. */
#define GS_STATIC_SCRATCH_BYTES (64u << 20)

gs_status gs_search_static(const gs_index* index, const int32_t* q_indptr, const int32_t* q_terms,
                           const float* q_w, int32_t batch, int64_t q_nnz, int32_t k, int32_t* out_ids,
                           void* out_scores, const gs_search_opts* opts, gs_stream_t stream);

/* Synchronises `stream`, then returns in *flags the GS_FLAG_* bits that the
 * last gs_search_static on the current device raised (the first word of the
 * fixed scratch array).  Allocates nothing. */
gs_status gs_search_static_flags(gs_stream_t stream, uint32_t* flags);

/* --- misc (library plumbing; the paper has no counterpart) --------------- */

/* a static string naming the status; never NULL */
const char* gs_status_str(gs_status status);
/* the CUDA error string of the last GS_ERR_CUDA on this host thread */
const char* gs_last_cuda_error(void);
int32_t gs_version(void); /* major * 10000 + minor * 100 + patch */
/* number of CUDA kernels this library has launched in the process so far */
int64_t gs_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* GPUSPARSE_H */
