// Batch runner: uneven query batches served from captured CUDA graphs, with
// tile shapes picked by a built-in autotuner.
//
// Batches are padded to power-of-two buckets (padding rows are empty
// queries, whose results are never copied out).  The first batch of each
// (bucket, k) is used to time a list of candidate doc-tiled plans — tile
// length T, queries per group G, sample stride R, dense head on or off, batch
// in the caller's order or regrouped by shared tail terms — the
// grid-search analogue of the paper's BLOCK_PL tuning (Sec. 5.2); the fastest
// plan's whole gs_search (prep, scoring, top-k) is captured once into a CUDA
// graph and every later batch of that bucket replays it with one launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "gs_internal.cuh"

struct gs_runner {
  const gs_index* ix = nullptr;
  int32_t max_batch = 0;  // a power of two
  int64_t max_q_nnz = 0;
  int32_t max_k = 0;
  int32_t autotune = 1;
  gs_search_opts base{};
  // device buffers
  int32_t* d_indptr = nullptr;
  int32_t* d_terms = nullptr;
  float* d_w = nullptr;
  int32_t* d_ids = nullptr;
  void* d_scores = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // pinned staging
  int32_t* h_indptr = nullptr;
  int32_t* h_terms = nullptr;
  float* h_w = nullptr;
  uint32_t* h_flags = nullptr;  // flag word of the last search
  // graphs are captured and replayed on the runner's own stream: capture is
  // not possible on the legacy default stream a caller may pass
  cudaStream_t own = nullptr;
  cudaEvent_t dep = nullptr;
  struct Entry {
    gs_search_opts opts{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    float tuned_ms = 0.f;
    int64_t replays = 0;
  };
  std::map<std::pair<int, int>, Entry> entries;
  std::mutex mu;
};

namespace {

int pow2_at_least(int v) {
  int b = 1;
  while (b < v) b <<= 1;
  return b;
}

// candidate doc-tiled plans for a bucket (shared memory holds G x T scores)
std::vector<gs_search_opts> candidates(const gs_index* ix, const gs_search_opts& base, int bucket) {
  std::vector<gs_search_opts> out;
  if (!ix->seg) {
    gs_search_opts o = base;
    o.algo = GS_ALGO_TERM_PARALLEL;
    for (int chunk : {16, 32, 64}) {
      o.chunk_blocks = chunk;
      out.push_back(o);
    }
    return out;
  }
  const int T0 = ix->tile_docs;
  for (int T = T0; T <= 4096; T *= 2) {
    for (int G : {4, 8, 16}) {
      if ((int64_t)G * T > 16384) continue;
      for (int head : {0, -1}) {
        if (head == 0 && (G != 16 || ix->head_H == 0)) continue;
        // groups larger than the bucket only for the dense head (its group is
        // fixed at 16 queries, and it can pay even half-filled)
        if (G > bucket && G != 4 && head != 0) continue;
        for (int R : {32, 64, 128}) {
          for (int qo : {-1, 1}) {  // caller's order, or regrouped by shared tail terms
            if (qo == 1 && (G < 8 || bucket < 2 * G)) continue;
            gs_search_opts o = base;
            o.algo = GS_ALGO_DOC_TILED;
            o.tile_docs = T;
            o.group_queries = G;
            o.use_head = head;
            o.sample_stride = R;
            o.query_order = qo;
            o.stage_events = nullptr;
            out.push_back(o);
          }
        }
      }
    }
  }
  return out;
}

gs_status launch_entry(gs_runner* r, int bucket, int k, cudaStream_t s, gs_runner::Entry** out) {
  auto key = std::make_pair(bucket, k);
  auto it = r->entries.find(key);
  if (it != r->entries.end()) {
    *out = &it->second;
    return GS_OK;
  }
  gs_runner::Entry e;
  e.opts = r->base;
  e.opts.stage_events = nullptr;
  if (r->autotune) {
    // time every candidate on this batch (already in the device buffers)
    cudaEvent_t a, b;
    GS_CUDA_TRY(cudaEventCreate(&a));
    GS_CUDA_TRY(cudaEventCreate(&b));
    float best = 1e30f;
    for (const gs_search_opts& o : candidates(r->ix, r->base, bucket)) {
      size_t need = 0;
      if (gs_search_workspace_size(r->ix, bucket, r->max_q_nnz, k, &o, 0, &need) != GS_OK || need > r->ws_bytes)
        continue;
      float ms = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        GS_CUDA_TRY(cudaEventRecord(a, s));
        gs_status st = gs_search(r->ix, r->d_indptr, r->d_terms, r->d_w, bucket, r->max_q_nnz, k, r->d_ids,
                                 r->d_scores, r->ws, r->ws_bytes, &o, reinterpret_cast<gs_stream_t>(s));
        if (st != GS_OK) break;
        GS_CUDA_TRY(cudaEventRecord(b, s));
        GS_CUDA_TRY(cudaEventSynchronize(b));
        float t = 0.f;
        GS_CUDA_TRY(cudaEventElapsedTime(&t, a, b));
        ms = std::min(ms, t);
      }
      if (ms < best) {
        best = ms;
        e.opts = o;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    e.tuned_ms = best;
  }
  // capture the chosen plan's whole search
  GS_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  gs_status st = gs_search(r->ix, r->d_indptr, r->d_terms, r->d_w, bucket, r->max_q_nnz, k, r->d_ids, r->d_scores,
                           r->ws, r->ws_bytes, &e.opts, reinterpret_cast<gs_stream_t>(s));
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (st != GS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ce != cudaSuccess) {
    gs::set_cuda_error(ce);
    return GS_ERR_CUDA;
  }
  e.graph = g;
  GS_CUDA_TRY(cudaGraphInstantiate(&e.exec, g, 0));
  auto res = r->entries.emplace(key, e);
  *out = &res.first->second;
  return GS_OK;
}

void free_runner(gs_runner* r) {
  if (!r) return;
  for (auto& kv : r->entries) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  cudaFree(r->d_indptr);
  cudaFree(r->d_terms);
  cudaFree(r->d_w);
  cudaFree(r->d_ids);
  cudaFree(r->d_scores);
  cudaFree(r->ws);
  cudaFreeHost(r->h_indptr);
  cudaFreeHost(r->h_terms);
  cudaFreeHost(r->h_w);
  cudaFreeHost(r->h_flags);
  if (r->dep) cudaEventDestroy(r->dep);
  if (r->own) cudaStreamDestroy(r->own);
  delete r;
}

}  // namespace

extern "C" gs_status gs_runner_create(const gs_index* index, int32_t max_batch, int64_t max_q_nnz, int32_t max_k,
                                      const gs_search_opts* opts, int32_t autotune, gs_runner** out) {
  if (!out) return GS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!index || max_batch < 1 || max_q_nnz < 1 || max_q_nnz > INT32_MAX - 1 || max_k < 1) return GS_ERR_INVALID_ARG;
  if (max_k > GS_MAX_K) return GS_ERR_UNSUPPORTED;
  if ((int64_t)max_k > index->N) return GS_ERR_INVALID_ARG;
  gs_runner* r = new gs_runner();
  r->ix = index;
  r->max_batch = pow2_at_least(max_batch);
  r->max_q_nnz = max_q_nnz;
  r->max_k = max_k;
  r->autotune = autotune ? 1 : 0;
  if (opts) r->base = *opts;
  r->base.stage_events = nullptr;
  // workspace: the largest any candidate plan needs at the top bucket
  size_t need = 0;
  {
    std::vector<gs_search_opts> cands = candidates(index, r->base, r->max_batch);
    cands.push_back(r->base);
    for (const gs_search_opts& o : cands) {
      size_t n = 0;
      for (int b = 1; b <= r->max_batch; b <<= 1)
        if (gs_search_workspace_size(index, b, max_q_nnz, max_k, &o, 0, &n) == GS_OK) need = std::max(need, n);
    }
  }
  cudaError_t e = cudaSuccess;
  const size_t B1 = (size_t)r->max_batch;
  if ((e = cudaMalloc(&r->d_indptr, sizeof(int32_t) * (B1 + 1))) != cudaSuccess ||
      (e = cudaMalloc(&r->d_terms, sizeof(int32_t) * max_q_nnz)) != cudaSuccess ||
      (e = cudaMalloc(&r->d_w, sizeof(float) * max_q_nnz)) != cudaSuccess ||
      (e = cudaMalloc(&r->d_ids, sizeof(int32_t) * B1 * max_k)) != cudaSuccess ||
      (e = cudaMalloc(&r->d_scores, sizeof(uint32_t) * B1 * max_k)) != cudaSuccess ||
      (e = cudaMalloc(&r->ws, need)) != cudaSuccess ||
      (e = cudaMallocHost(&r->h_indptr, sizeof(int32_t) * (B1 + 1))) != cudaSuccess ||
      (e = cudaMallocHost(&r->h_terms, sizeof(int32_t) * max_q_nnz)) != cudaSuccess ||
      (e = cudaMallocHost(&r->h_w, sizeof(float) * max_q_nnz)) != cudaSuccess ||
      (e = cudaMallocHost(&r->h_flags, sizeof(uint32_t))) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&r->own, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&r->dep, cudaEventDisableTiming)) != cudaSuccess) {
    gs::set_cuda_error(e);
    free_runner(r);
    return e == cudaErrorMemoryAllocation ? GS_ERR_OUT_OF_MEMORY : GS_ERR_CUDA;
  }
  r->ws_bytes = need;
  *out = r;
  return GS_OK;
}

extern "C" gs_status gs_runner_search(gs_runner* r, const int32_t* h_q_indptr, const int32_t* h_q_terms,
                                      const float* h_q_w, int32_t batch, int32_t k, int32_t* h_out_ids,
                                      void* h_out_scores, gs_stream_t stream) {
  if (!r || !h_q_indptr || batch < 1 || batch > r->max_batch || k < 1 || k > r->max_k || !h_out_ids ||
      !h_out_scores)
    return GS_ERR_INVALID_ARG;
  const int64_t nnz = h_q_indptr[batch];
  if (h_q_indptr[0] != 0 || nnz < 0 || nnz > r->max_q_nnz || (nnz > 0 && (!h_q_terms || !h_q_w)))
    return GS_ERR_INVALID_ARG;
  for (int32_t q = 0; q < batch; ++q)
    if (h_q_indptr[q + 1] < h_q_indptr[q]) return GS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(r->mu);
  // work already queued on the caller's stream comes first
  GS_CUDA_TRY(cudaEventRecord(r->dep, reinterpret_cast<cudaStream_t>(stream)));
  cudaStream_t s = r->own;
  GS_CUDA_TRY(cudaStreamWaitEvent(s, r->dep, 0));
  const int bucket = pow2_at_least(batch);
  // padded batch: queries past `batch` are empty
  std::memcpy(r->h_indptr, h_q_indptr, sizeof(int32_t) * (batch + 1));
  for (int q = batch + 1; q <= bucket; ++q) r->h_indptr[q] = (int32_t)nnz;
  if (nnz > 0) {
    std::memcpy(r->h_terms, h_q_terms, sizeof(int32_t) * nnz);
    std::memcpy(r->h_w, h_q_w, sizeof(float) * nnz);
  }
  GS_CUDA_TRY(cudaMemcpyAsync(r->d_indptr, r->h_indptr, sizeof(int32_t) * (bucket + 1), cudaMemcpyHostToDevice, s));
  if (nnz > 0) {
    GS_CUDA_TRY(cudaMemcpyAsync(r->d_terms, r->h_terms, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
    GS_CUDA_TRY(cudaMemcpyAsync(r->d_w, r->h_w, sizeof(float) * nnz, cudaMemcpyHostToDevice, s));
  }
  gs_runner::Entry* e = nullptr;
  gs_status st = launch_entry(r, bucket, k, s, &e);
  if (st != GS_OK) return st;
  GS_CUDA_TRY(cudaGraphLaunch(e->exec, s));
  gs::count_launches(1);
  ++e->replays;
  GS_CUDA_TRY(cudaMemcpyAsync(h_out_ids, r->d_ids, sizeof(int32_t) * (size_t)batch * k, cudaMemcpyDeviceToHost, s));
  GS_CUDA_TRY(
      cudaMemcpyAsync(h_out_scores, r->d_scores, sizeof(uint32_t) * (size_t)batch * k, cudaMemcpyDeviceToHost, s));
  // the search's flag word leads the workspace
  GS_CUDA_TRY(cudaMemcpyAsync(r->h_flags, r->ws, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA_TRY(cudaStreamSynchronize(s));
  return gs::flags_status(*r->h_flags);
}

extern "C" gs_status gs_runner_plan(gs_runner* r, int32_t batch, int32_t k, gs_search_opts* out_opts,
                                    float* out_tuned_ms) {
  if (!r || !out_opts) return GS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(r->mu);
  auto it = r->entries.find(std::make_pair(pow2_at_least(std::max(batch, 1)), k));
  if (it == r->entries.end()) return GS_ERR_INVALID_ARG;
  *out_opts = it->second.opts;
  if (out_tuned_ms) *out_tuned_ms = it->second.tuned_ms;
  return GS_OK;
}

extern "C" void gs_runner_free(gs_runner* r) { free_runner(r); }
