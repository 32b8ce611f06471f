// Serving loop with continuous batching (the paper's future-work item 3,
// Sec. 8: streaming query batching with adaptive accumulation).
//
// Requests (one sparse query, its k and its target index) are queued on the
// host.  A lane is one admission slot: a CUDA stream, a search workspace
// (the score-row memory of a batch), device and pinned host buffers.  The
// number of lanes follows from the workspace budget, so requests are admitted
// as score-buffer memory frees up.  A scheduler thread forms a batch from the
// pending requests of one index whenever a lane is free — the oldest request
// first, then every pending request of that index that fits — and enqueues
// copy, search and copy-back on the lane's stream; batches of different lanes
// run concurrently on the device.  One completion thread per lane waits for
// its batch, hands every request the first k entries of the batch's top-k
// (the batch runs with the largest k of its requests; the order is total, so
// a prefix of the top-K list is the top-k list) and frees the lane.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gs_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  int32_t index_id = 0;
  int32_t k = 0;
  std::vector<int32_t> terms;
  std::vector<float> weights;
  Clock::time_point arrival;
  std::vector<int32_t> ids;
  std::vector<uint32_t> scores;
  double latency_us = 0.0;
  bool done = false;
  gs_status status = GS_OK;
};

struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int32_t* d_indptr = nullptr;
  int32_t* d_terms = nullptr;
  float* d_w = nullptr;
  int32_t* d_ids = nullptr;
  uint32_t* d_scores = nullptr;
  int32_t* h_indptr = nullptr;
  int32_t* h_terms = nullptr;
  float* h_w = nullptr;
  int32_t* h_ids = nullptr;
  uint32_t* h_scores = nullptr;
  uint32_t* h_flags = nullptr;  // the batch's flag word
  // the batch in flight
  std::vector<std::shared_ptr<Request>> batch;
  int32_t batch_k = 0;
  bool busy = false;
  gs_status launch_status = GS_OK;
  std::thread completer;
};

}  // namespace

struct gs_server {
  std::vector<const gs_index*> indexes;
  gs_server_config cfg{};
  int device = 0;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::mutex mu;
  std::condition_variable cv_sched;  // requests arrived / a lane freed / stop
  std::condition_variable cv_lane;   // a lane got a batch / stop
  std::condition_variable cv_done;   // a request completed
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<int64_t, std::shared_ptr<Request>> tickets;
  int64_t next_ticket = 1;
  bool stop = false;
  std::thread scheduler;
  // statistics
  int64_t completed = 0;
  int64_t batches = 0;
  int64_t batched_queries = 0;
  int32_t max_in_flight = 0;
};

namespace {

void free_lane(Lane* L) {
  cudaFree(L->ws);
  cudaFree(L->d_indptr);
  cudaFree(L->d_terms);
  cudaFree(L->d_w);
  cudaFree(L->d_ids);
  cudaFree(L->d_scores);
  cudaFreeHost(L->h_indptr);
  cudaFreeHost(L->h_terms);
  cudaFreeHost(L->h_w);
  cudaFreeHost(L->h_ids);
  cudaFreeHost(L->h_scores);
  cudaFreeHost(L->h_flags);
  if (L->done_ev) cudaEventDestroy(L->done_ev);
  if (L->stream) cudaStreamDestroy(L->stream);
}

// Enqueue one batch on a lane (called with the server mutex held).
gs_status launch_batch(gs_server* S, Lane* L) {
  const int B = (int)L->batch.size();
  const gs_index* ix = S->indexes[L->batch[0]->index_id];
  int32_t k = 0;
  int64_t nnz = 0;
  L->h_indptr[0] = 0;
  for (int i = 0; i < B; ++i) {
    const Request& r = *L->batch[i];
    k = std::max(k, r.k);
    std::memcpy(L->h_terms + nnz, r.terms.data(), sizeof(int32_t) * r.terms.size());
    std::memcpy(L->h_w + nnz, r.weights.data(), sizeof(float) * r.weights.size());
    nnz += (int64_t)r.terms.size();
    L->h_indptr[i + 1] = (int32_t)nnz;
  }
  L->batch_k = k;
  cudaStream_t s = L->stream;
  GS_CUDA_TRY(cudaSetDevice(S->device));
  GS_CUDA_TRY(cudaMemcpyAsync(L->d_indptr, L->h_indptr, sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, s));
  if (nnz > 0) {
    GS_CUDA_TRY(cudaMemcpyAsync(L->d_terms, L->h_terms, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
    GS_CUDA_TRY(cudaMemcpyAsync(L->d_w, L->h_w, sizeof(float) * nnz, cudaMemcpyHostToDevice, s));
  }
  gs_status st = gs_search(ix, L->d_indptr, L->d_terms, L->d_w, B, S->cfg.max_q_nnz, k, L->d_ids, L->d_scores, L->ws,
                           L->ws_bytes, &S->cfg.opts, reinterpret_cast<gs_stream_t>(s));
  if (st != GS_OK) return st;
  GS_CUDA_TRY(cudaMemcpyAsync(L->h_ids, L->d_ids, sizeof(int32_t) * (size_t)B * k, cudaMemcpyDeviceToHost, s));
  GS_CUDA_TRY(cudaMemcpyAsync(L->h_scores, L->d_scores, sizeof(uint32_t) * (size_t)B * k, cudaMemcpyDeviceToHost, s));
  GS_CUDA_TRY(cudaMemcpyAsync(L->h_flags, L->ws, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));  // flag word
  GS_CUDA_TRY(cudaEventRecord(L->done_ev, s));
  return GS_OK;
}

void scheduler_loop(gs_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (true) {
    Lane* free_lane_p = nullptr;
    S->cv_sched.wait(lock, [&] {
      if (S->stop) return true;
      if (S->queue.empty()) return false;
      for (auto& L : S->lanes)
        if (!L->busy) return true;
      return false;
    });
    if (S->stop) return;
    for (auto& L : S->lanes)
      if (!L->busy) {
        free_lane_p = L.get();
        break;
      }
    // optional short accumulation window once the first request waits
    if (S->cfg.max_wait_us > 0 && (int)S->queue.size() < S->cfg.max_batch) {
      const auto deadline = S->queue.front()->arrival + std::chrono::microseconds(S->cfg.max_wait_us);
      S->cv_sched.wait_until(lock, deadline, [&] { return S->stop || (int)S->queue.size() >= S->cfg.max_batch; });
      if (S->stop) return;
    }
    // batch: the oldest request's index, then every pending request of that
    // index that fits the lane (batch size and term capacity)
    const int32_t target = S->queue.front()->index_id;
    int64_t nnz = 0;
    for (auto it = S->queue.begin(); it != S->queue.end() && (int)free_lane_p->batch.size() < S->cfg.max_batch;) {
      auto& r = *it;
      if (r->index_id == target && nnz + (int64_t)r->terms.size() <= S->cfg.max_q_nnz) {
        nnz += (int64_t)r->terms.size();
        free_lane_p->batch.push_back(r);
        it = S->queue.erase(it);
      } else {
        ++it;
      }
    }
    free_lane_p->busy = true;
    free_lane_p->launch_status = launch_batch(S, free_lane_p);
    int in_flight = 0;
    for (auto& L : S->lanes) in_flight += L->busy ? 1 : 0;
    S->max_in_flight = std::max(S->max_in_flight, in_flight);
    S->batches += 1;
    S->batched_queries += (int64_t)free_lane_p->batch.size();
    S->cv_lane.notify_all();
  }
}

void completer_loop(gs_server* S, Lane* L) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (true) {
    S->cv_lane.wait(lock, [&] { return S->stop || (L->busy && !L->batch.empty()); });
    if (S->stop && !L->busy) return;
    if (S->stop && L->busy && L->launch_status != GS_OK) return;
    gs_status st = L->launch_status;
    if (st == GS_OK) {
      lock.unlock();
      cudaError_t e = cudaEventSynchronize(L->done_ev);
      lock.lock();
      if (e != cudaSuccess) {
        gs::set_cuda_error(e);
        st = GS_ERR_CUDA;
      } else if (gs::flags_status(*L->h_flags) != GS_OK) {
        st = gs::flags_status(*L->h_flags);  // submit validates every query: not expected
      }
    }
    const auto now = Clock::now();
    const int K = L->batch_k;
    for (size_t i = 0; i < L->batch.size(); ++i) {
      Request& r = *L->batch[i];
      r.status = st;
      if (st == GS_OK) {
        r.ids.assign(L->h_ids + i * K, L->h_ids + i * K + r.k);
        r.scores.assign(L->h_scores + i * K, L->h_scores + i * K + r.k);
      }
      r.latency_us = std::chrono::duration<double, std::micro>(now - r.arrival).count();
      r.done = true;
      S->completed += 1;
    }
    L->batch.clear();
    L->busy = false;
    S->cv_done.notify_all();
    S->cv_sched.notify_all();
    if (S->stop) return;
  }
}

}  // namespace

extern "C" gs_status gs_server_create(const gs_index* const* indexes, int32_t n_indexes,
                                      const gs_server_config* cfg, gs_server** out) {
  if (!out) return GS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!indexes || n_indexes < 1 || !cfg || cfg->max_batch < 1 || cfg->max_q_nnz < 1 || cfg->max_k < 1)
    return GS_ERR_INVALID_ARG;
  if (cfg->max_k > GS_MAX_K) return GS_ERR_UNSUPPORTED;
  auto S = std::make_unique<gs_server>();
  S->cfg = *cfg;
  S->cfg.opts.stage_events = nullptr;
  for (int i = 0; i < n_indexes; ++i) {
    if (!indexes[i] || (int64_t)cfg->max_k > indexes[i]->N) return GS_ERR_INVALID_ARG;
    S->indexes.push_back(indexes[i]);
  }
  GS_CUDA_TRY(cudaGetDevice(&S->device));
  // one lane = one batch's workspace on the most demanding index
  size_t ws = 0;
  for (const gs_index* ix : S->indexes) {
    size_t n = 0;
    gs_status st = gs_search_workspace_size(ix, cfg->max_batch, cfg->max_q_nnz, cfg->max_k, &S->cfg.opts, 0, &n);
    if (st != GS_OK) return st;
    ws = std::max(ws, n);
  }
  int lanes = std::max(1, cfg->lanes);
  if (cfg->workspace_budget_bytes > 0)
    lanes = (int)std::max<int64_t>(1, std::min<int64_t>(lanes, cfg->workspace_budget_bytes / (int64_t)ws));
  for (int i = 0; i < lanes; ++i) {
    auto L = std::make_unique<Lane>();
    cudaError_t e = cudaSuccess;
    const size_t B = cfg->max_batch, Q = cfg->max_q_nnz, K = cfg->max_k;
    if ((e = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&L->done_ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMalloc(&L->ws, ws)) != cudaSuccess || (e = cudaMalloc(&L->d_indptr, 4 * (B + 1))) != cudaSuccess ||
        (e = cudaMalloc(&L->d_terms, 4 * Q)) != cudaSuccess || (e = cudaMalloc(&L->d_w, 4 * Q)) != cudaSuccess ||
        (e = cudaMalloc(&L->d_ids, 4 * B * K)) != cudaSuccess || (e = cudaMalloc(&L->d_scores, 4 * B * K)) != cudaSuccess ||
        (e = cudaMallocHost(&L->h_indptr, 4 * (B + 1))) != cudaSuccess ||
        (e = cudaMallocHost(&L->h_terms, 4 * Q)) != cudaSuccess || (e = cudaMallocHost(&L->h_w, 4 * Q)) != cudaSuccess ||
        (e = cudaMallocHost(&L->h_ids, 4 * B * K)) != cudaSuccess ||
        (e = cudaMallocHost(&L->h_scores, 4 * B * K)) != cudaSuccess ||
        (e = cudaMallocHost(&L->h_flags, 4)) != cudaSuccess) {
      gs::set_cuda_error(e);
      free_lane(L.get());
      for (auto& l : S->lanes) free_lane(l.get());
      return e == cudaErrorMemoryAllocation ? GS_ERR_OUT_OF_MEMORY : GS_ERR_CUDA;
    }
    L->ws_bytes = ws;
    S->lanes.push_back(std::move(L));
  }
  gs_server* raw = S.release();
  for (auto& L : raw->lanes) L->completer = std::thread(completer_loop, raw, L.get());
  raw->scheduler = std::thread(scheduler_loop, raw);
  *out = raw;
  return GS_OK;
}

extern "C" gs_status gs_server_submit(gs_server* S, int32_t index_id, const int32_t* terms, const float* weights,
                                      int32_t nnz, int32_t k, int64_t* ticket) {
  if (!S || !ticket || index_id < 0 || index_id >= (int32_t)S->indexes.size() || nnz < 0 ||
      nnz > S->cfg.max_q_nnz || k < 1 || k > S->cfg.max_k || (nnz > 0 && (!terms || !weights)))
    return GS_ERR_INVALID_ARG;
  if ((int64_t)k > S->indexes[index_id]->N) return GS_ERR_INVALID_ARG;
  // the query itself: term ids in [0, V) and finite weights
  const int32_t V = S->indexes[index_id]->V;
  for (int32_t i = 0; i < nnz; ++i)
    if (terms[i] < 0 || terms[i] >= V || !std::isfinite(weights[i])) return GS_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
  r->index_id = index_id;
  r->k = k;
  r->terms.assign(terms, terms + nnz);
  r->weights.assign(weights, weights + nnz);
  r->arrival = Clock::now();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) return GS_ERR_INVALID_ARG;
    r->ticket = S->next_ticket++;
    S->tickets.emplace(r->ticket, r);
    S->queue.push_back(r);
  }
  S->cv_sched.notify_one();
  *ticket = r->ticket;
  return GS_OK;
}

extern "C" gs_status gs_server_wait(gs_server* S, int64_t ticket, int32_t* out_ids, void* out_scores,
                                    int64_t timeout_us, double* latency_us) {
  if (!S || !out_ids || !out_scores) return GS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return GS_ERR_INVALID_ARG;
  std::shared_ptr<Request> r = it->second;
  const bool ok = S->cv_done.wait_for(lock, std::chrono::microseconds(std::max<int64_t>(timeout_us, 0)),
                                      [&] { return r->done; });
  if (!ok) return GS_ERR_TIMEOUT;  // the request stays queued; wait again later
  S->tickets.erase(ticket);
  if (r->status != GS_OK) return r->status;
  std::memcpy(out_ids, r->ids.data(), sizeof(int32_t) * r->ids.size());
  std::memcpy(out_scores, r->scores.data(), sizeof(uint32_t) * r->scores.size());
  if (latency_us) *latency_us = r->latency_us;
  return GS_OK;
}

extern "C" gs_status gs_server_stats_get(gs_server* S, gs_server_stats* out) {
  if (!S || !out) return GS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->lanes = (int32_t)S->lanes.size();
  out->max_in_flight = S->max_in_flight;
  out->completed = S->completed;
  out->batches = S->batches;
  out->batched_queries = S->batched_queries;
  out->queued = (int64_t)S->queue.size();
  out->lane_workspace_bytes = S->lanes.empty() ? 0 : (int64_t)S->lanes[0]->ws_bytes;
  return GS_OK;
}

extern "C" void gs_server_destroy(gs_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_sched.notify_all();
  S->cv_lane.notify_all();
  S->cv_done.notify_all();
  if (S->scheduler.joinable()) S->scheduler.join();
  for (auto& L : S->lanes) {
    if (L->completer.joinable()) L->completer.join();
  }
  for (auto& L : S->lanes) {
    if (L->stream) cudaStreamSynchronize(L->stream);
    free_lane(L.get());
  }
  delete S;
}
