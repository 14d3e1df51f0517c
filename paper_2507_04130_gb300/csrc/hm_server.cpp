// hm_server.cpp -- a query server over one resident target graph (host runtime).
//
// Queries (pattern + mode + whether rows are wanted) are submitted from any
// thread and return immediately with an id.  A fixed number of dispatcher
// slots, each a host thread with its own CUDA stream, serve them: whenever a
// slot is free it takes every waiting query that the device-memory budget
// admits (up to max_batch), runs them as ONE batch (hm_count_batch, then
// hm_enumerate_batch for the queries that want rows and whose rows fit the
// budget), copies the rows to host memory and completes the queries.  Queries
// arriving while batches are on the GPU join the next free slot's batch, and
// batches of different slots run concurrently on the device (continuous
// batching at launch granularity).
//
// Admission: a query reserves the worst-case device memory of its depth-2
// states -- two seed queues of (int2 + pattern id) per target arc, 24 B x m --
// plus a fixed share for the control block and the donation queue; rows are
// reserved from the count before enumeration, and a query whose rows do not
// fit the remaining budget is answered with its count only (rows_dropped).
// Latency is measured from submit to completion on the host clock.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hm_internal.cuh"

namespace {

using clock_t_ = std::chrono::steady_clock;

struct Query {
  uint64_t id = 0;
  hm_pattern *pattern = nullptr;
  int32_t mode = 0;
  int32_t want_rows = 0;
  int32_t k = 0;
  clock_t_::time_point t_submit;
  // results
  std::atomic<int32_t> done{0};
  hm_status status = HM_OK;
  uint64_t count = 0;
  int32_t rows_dropped = 0;
  std::vector<int32_t> rows;  // host copy
  double latency_ms = 0;
  uint64_t reserved = 0;
};

}  // namespace

struct hm_server {
  const hm_graph *g = nullptr;
  int32_t device = 0;
  int32_t nslots = 1;
  int32_t max_batch = 64;
  uint64_t mem_budget = 0;
  uint64_t per_query_bytes = 0;

  std::mutex mu;
  std::condition_variable cv;      // work arrived / memory freed / shutdown
  std::condition_variable done_cv; // a query completed
  std::deque<std::shared_ptr<Query>> waiting;
  std::unordered_map<uint64_t, std::shared_ptr<Query>> all;
  uint64_t next_id = 1;
  uint64_t in_use = 0;            // reserved device bytes
  bool stop = false;
  std::vector<std::thread> threads;

  // counters
  uint64_t batches = 0, completed = 0, max_inflight_batches = 0, inflight_batches = 0;
  uint64_t rows_dropped = 0;
};

namespace {

void serve_slot(hm_server *S, int slot) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  for (;;) {
    std::vector<std::shared_ptr<Query>> batch;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // wake for an admissible batch, or (when stopping) once nothing waits;
      // while stopping, queries still waiting for memory are drained as usual
      S->cv.wait(lk, [&] {
        const bool admit = S->in_use + S->per_query_bytes <= S->mem_budget;
        return S->stop ? (S->waiting.empty() || admit) : (!S->waiting.empty() && admit);
      });
      if (S->stop && S->waiting.empty()) break;
      while (!S->waiting.empty() && (int32_t)batch.size() < S->max_batch &&
             S->in_use + S->per_query_bytes <= S->mem_budget) {
        auto q = S->waiting.front();
        S->waiting.pop_front();
        q->reserved = S->per_query_bytes;
        S->in_use += q->reserved;
        batch.push_back(q);
      }
      if (batch.empty()) continue;
      S->batches++;
      S->inflight_batches++;
      S->max_inflight_batches = std::max(S->max_inflight_batches, S->inflight_batches);
    }
    const int32_t nb = (int32_t)batch.size();
    std::vector<const hm_pattern *> pats(nb);
    std::vector<int32_t> modes(nb);
    std::vector<uint64_t> counts(nb, 0);
    for (int32_t i = 0; i < nb; ++i) {
      pats[i] = batch[i]->pattern;
      modes[i] = batch[i]->mode;
    }
    hm_status st = hm_count_batch(S->g, pats.data(), modes.data(), nb, counts.data(), stream);
    if (st == HM_OK) {
      for (int32_t i = 0; i < nb; ++i) batch[i]->count = counts[i];
      // rows: reserve what the counts say, enumerate the queries that fit
      std::vector<int32_t> rows_idx;
      uint64_t need = 0;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        for (int32_t i = 0; i < nb; ++i) {
          if (!batch[i]->want_rows) continue;
          const uint64_t b = counts[i] * (uint64_t)batch[i]->k * sizeof(int32_t);
          if (S->in_use + need + b <= S->mem_budget) {
            need += b;
            rows_idx.push_back(i);
          } else {
            batch[i]->rows_dropped = 1;
            S->rows_dropped++;
          }
        }
        S->in_use += need;
      }
      if (!rows_idx.empty()) {
        const int32_t nr = (int32_t)rows_idx.size();
        std::vector<const hm_pattern *> rp(nr);
        std::vector<int32_t> rm(nr);
        std::vector<uint64_t> off(nr + 1, 0), rc(nr, 0);
        for (int32_t j = 0; j < nr; ++j) {
          const auto &q = batch[rows_idx[j]];
          rp[j] = q->pattern;
          rm[j] = q->mode;
          off[j + 1] = off[j] + q->count * (uint64_t)q->k;
        }
        int32_t *d_rows = nullptr;
        cudaError_t e = cudaMallocAsync((void **)&d_rows, sizeof(int32_t) * std::max<uint64_t>(off[nr], 1), stream);
        if (e != cudaSuccess) {
          (void)cudaGetLastError();
          st = HM_ERR_OOM;
        } else {
          st = hm_enumerate_batch(S->g, rp.data(), rm.data(), nr, d_rows, off.data(), rc.data(), stream);
          if (st == HM_OK) {
            for (int32_t j = 0; j < nr; ++j) {
              auto &q = batch[rows_idx[j]];
              q->rows.resize(q->count * (uint64_t)q->k);
              if (!q->rows.empty() &&
                  cudaMemcpyAsync(q->rows.data(), d_rows + off[j], sizeof(int32_t) * q->rows.size(),
                                  cudaMemcpyDeviceToHost, stream) != cudaSuccess)
                st = HM_ERR_CUDA;
            }
            if (cudaStreamSynchronize(stream) != cudaSuccess) st = HM_ERR_CUDA;
          }
          cudaFreeAsync(d_rows, stream);
        }
      }
      std::lock_guard<std::mutex> lk(S->mu);
      S->in_use -= need;
    }
    const auto t_end = clock_t_::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto &q : batch) {
        q->status = st;
        q->latency_ms = std::chrono::duration<double, std::milli>(t_end - q->t_submit).count();
        S->in_use -= q->reserved;
        q->reserved = 0;
        q->done.store(1);
        S->completed++;
      }
      S->inflight_batches--;
    }
    S->cv.notify_all();
    S->done_cv.notify_all();
  }
  cudaStreamSynchronize(stream);
  cudaStreamDestroy(stream);
}

}  // namespace

extern "C" hm_status hm_server_create(const hm_graph *g, int32_t nslots, int32_t max_batch,
                                      uint64_t mem_budget, hm_server **out) {
  if (!g || !out || nslots < 1 || nslots > 64 || max_batch < 1) return HM_ERR_ARG;
  auto *S = new hm_server();
  S->g = g;
  S->device = g->device;
  S->nslots = nslots;
  S->max_batch = max_batch;
  S->per_query_bytes = 24ull * (uint64_t)std::max<int64_t>(g->m, 1) + (8u << 20);
  // default: every slot full of queries, plus as much again for their rows
  S->mem_budget = mem_budget ? mem_budget : 2 * S->per_query_bytes * (uint64_t)max_batch * nslots;
  if (S->mem_budget < S->per_query_bytes) {
    delete S;
    return HM_ERR_ARG;  // the budget cannot admit even one query
  }
  for (int32_t i = 0; i < nslots; ++i) S->threads.emplace_back(serve_slot, S, i);
  *out = S;
  return HM_OK;
}

extern "C" hm_status hm_server_submit(hm_server *S, int32_t k, int32_t mp, const int32_t *src,
                                      const int32_t *dst, const int32_t *vlab, const int32_t *elab,
                                      int32_t mode, int32_t want_rows, uint64_t *qid) {
  if (!S || !qid || (mode != HM_MONO && mode != HM_INDUCED)) return HM_ERR_ARG;
  hm_pattern *p = nullptr;
  hm_status st = hm_load_pattern(k, mp, src, dst, vlab, elab, &p);
  if (st != HM_OK) return st;
  auto q = std::make_shared<Query>();
  q->pattern = p;
  q->mode = mode;
  q->want_rows = want_rows ? 1 : 0;
  q->k = k;
  q->t_submit = clock_t_::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      hm_free_pattern(p);
      return HM_ERR_ARG;
    }
    q->id = S->next_id++;
    S->all[q->id] = q;
    S->waiting.push_back(q);
  }
  S->cv.notify_one();
  *qid = q->id;
  return HM_OK;
}

extern "C" hm_status hm_server_poll(hm_server *S, uint64_t qid, int32_t wait, int32_t *done,
                                    uint64_t *count, double *latency_ms, int32_t *rows_dropped,
                                    const int32_t **rows, uint64_t *nrows) {
  if (!S || !done) return HM_ERR_ARG;
  std::shared_ptr<Query> q;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(qid);
    if (it == S->all.end()) return HM_ERR_ARG;
    q = it->second;
    if (wait) S->done_cv.wait(lk, [&] { return q->done.load() != 0; });
  }
  *done = q->done.load();
  if (!*done) return HM_OK;
  if (count) *count = q->count;
  if (latency_ms) *latency_ms = q->latency_ms;
  if (rows_dropped) *rows_dropped = q->rows_dropped;
  if (rows) *rows = q->rows.empty() ? nullptr : q->rows.data();
  if (nrows) *nrows = q->k ? q->rows.size() / (uint64_t)q->k : 0;
  return q->status;
}

extern "C" hm_status hm_server_release(hm_server *S, uint64_t qid) {
  if (!S) return HM_ERR_ARG;
  std::shared_ptr<Query> q;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(qid);
    if (it == S->all.end() || !it->second->done.load()) return HM_ERR_ARG;
    q = it->second;
    S->all.erase(it);
  }
  hm_free_pattern(q->pattern);
  q->pattern = nullptr;
  return HM_OK;
}

extern "C" hm_status hm_server_stats(hm_server *S, uint64_t *batches, uint64_t *completed,
                                     uint64_t *max_inflight_batches, uint64_t *rows_dropped) {
  if (!S) return HM_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (batches) *batches = S->batches;
  if (completed) *completed = S->completed;
  if (max_inflight_batches) *max_inflight_batches = S->max_inflight_batches;
  if (rows_dropped) *rows_dropped = S->rows_dropped;
  return HM_OK;
}

extern "C" void hm_server_destroy(hm_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto &t : S->threads) t.join();
  for (auto &kv : S->all)
    if (kv.second->pattern) hm_free_pattern(kv.second->pattern);
  delete S;
}
