// hm_server.cpp -- a query server over one resident target graph (host runtime).
//
// Queries (pattern + mode + whether rows are wanted) are submitted from any
// thread and return immediately with an id.  A fixed number of dispatcher
// slots, each a host thread with its own CUDA stream, serve them: whenever a
// slot is free it takes the waiting queries, in arrival order, that the
// device-memory budget admits (up to max_batch) and runs them as ONE batch;
// queries arriving while batches are on the GPU join the next free slot's
// batch, and batches of different slots run concurrently on the device
// (continuous batching at launch granularity).
//
// Admission by the device memory a query needs: its depth-2 states can be no
// more than the target arcs whose label and end labels fit its seeding arc
// (counted once per (source label, arc label, target label) when the server
// is created, from the graph's label-grouped directory), and each takes two
// seed-queue entries (12 B each, with the pattern id); the donation queue and
// control block (kBatchFixed) are charged once per batch.  The warps' DFS
// stacks live in shared memory and cost no device memory.
//
// One pass per batch: the rows of each query that wants them go to a region
// sized by a guess (row_guess rows, within the budget); the batched
// enumeration returns every count and keeps the sorted rows of the queries
// that fit.  Only a query whose count exceeds its guess runs again, with its
// exact size if the budget holds it, otherwise it is answered with its count
// alone (rows_dropped).  Latency is measured from submit to completion on the
// host clock.
#include <algorithm>
#include <atomic>
#include <map>
#include <tuple>
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
  uint64_t need = 0;  // device bytes to admit it (its seed queues)
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
  uint64_t row_guess = 1u << 18;  // rows a query's region holds on the first pass
  // arcs per (source label, arc label, target label)
  std::map<std::tuple<int32_t, int32_t, int32_t>, uint64_t> triples;

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

// Device memory a batch takes besides its queries' seed queues and rows: the
// donation queue, its sequence words and the control block.
constexpr uint64_t kBatchFixed = (12ull << 20);

void serve_slot(hm_server *S, int slot) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  for (;;) {
    std::vector<std::shared_ptr<Query>> batch;
    uint64_t held = 0;  // bytes this batch reserved at admission
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // the head query fits the budget, or nothing is running (a query larger
      // than the whole budget still runs, alone); while stopping, drain
      auto admissible = [&] {
        return !S->waiting.empty() &&
               (S->in_use == 0 || S->in_use + S->waiting.front()->need + kBatchFixed <= S->mem_budget);
      };
      S->cv.wait(lk, [&] { return admissible() || (S->stop && S->waiting.empty()); });
      if (S->stop && S->waiting.empty()) break;
      while (!S->waiting.empty() && (int32_t)batch.size() < S->max_batch) {
        auto q = S->waiting.front();
        const uint64_t add = q->need + (batch.empty() ? kBatchFixed : 0);
        if (!(S->in_use + add <= S->mem_budget || (S->in_use == 0 && batch.empty()))) break;
        S->waiting.pop_front();
        q->reserved = add;
        S->in_use += add;
        held += add;
        batch.push_back(q);
      }
      if (batch.empty()) continue;
      S->batches++;
      S->inflight_batches++;
      S->max_inflight_batches = std::max(S->max_inflight_batches, S->inflight_batches);
    }
    const int32_t nb = (int32_t)batch.size();
    hm::NvtxRange r_batch("hm.server_batch");
    std::vector<const hm_pattern *> pats(nb);
    std::vector<int32_t> modes(nb);
    std::vector<uint64_t> counts(nb, 0);
    bool any_rows = false;
    for (int32_t i = 0; i < nb; ++i) {
      pats[i] = batch[i]->pattern;
      modes[i] = batch[i]->mode;
      any_rows |= batch[i]->want_rows != 0;
    }
    hm_status st = HM_OK;
    if (!any_rows) {
      st = hm_count_batch(S->g, pats.data(), modes.data(), nb, counts.data(), stream);
      for (int32_t i = 0; i < nb && st == HM_OK; ++i) batch[i]->count = counts[i];
    } else {
      // one pass: rows into regions of row_guess rows (as many as the budget holds)
      uint64_t rows_bytes = 0;
      std::vector<uint64_t> off(nb + 1, 0);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        const uint64_t room = S->mem_budget > S->in_use ? S->mem_budget - S->in_use : 0;
        uint64_t want = 0;
        for (int32_t i = 0; i < nb; ++i)
          if (batch[i]->want_rows) want += S->row_guess * (uint64_t)batch[i]->k * sizeof(int32_t);
        const uint64_t guess = want <= room || want == 0 ? S->row_guess
                                                         : std::max<uint64_t>(1, S->row_guess * room / want);
        for (int32_t i = 0; i < nb; ++i)
          off[i + 1] = off[i] + (batch[i]->want_rows ? guess * (uint64_t)batch[i]->k : 0);
        rows_bytes = off[nb] * sizeof(int32_t);
        S->in_use += rows_bytes;
      }
      std::vector<uint8_t> fit(nb, 0);
      int32_t *d_rows = nullptr;
      cudaError_t e = cudaMallocAsync((void **)&d_rows, std::max<uint64_t>(rows_bytes, 16), stream);
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        st = HM_ERR_OOM;
      } else {
        st = hm::enumerate_batch_fit(S->g, pats.data(), modes.data(), nb, d_rows, off.data(), counts.data(),
                                     fit.data(), stream);
        if (st == HM_OK) {
          for (int32_t i = 0; i < nb; ++i) {
            auto &q = batch[i];
            q->count = counts[i];
            if (!q->want_rows || !fit[i] || !q->count) continue;
            q->rows.resize(q->count * (uint64_t)q->k);
            if (cudaMemcpyAsync(q->rows.data(), d_rows + off[i], sizeof(int32_t) * q->rows.size(),
                                cudaMemcpyDeviceToHost, stream) != cudaSuccess)
              st = HM_ERR_CUDA;
          }
          if (cudaStreamSynchronize(stream) != cudaSuccess) st = HM_ERR_CUDA;
        }
        cudaFreeAsync(d_rows, stream);
      }
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->in_use -= rows_bytes;
      }
      // a second pass, at the exact size, for the queries whose rows did not fit
      std::vector<int32_t> again;
      for (int32_t i = 0; i < nb && st == HM_OK; ++i)
        if (batch[i]->want_rows && !fit[i]) again.push_back(i);
      if (st == HM_OK && !again.empty()) {
        std::vector<int32_t> take;
        uint64_t need = 0;
        {
          std::lock_guard<std::mutex> lk(S->mu);
          for (int32_t i : again) {
            const uint64_t b = counts[i] * (uint64_t)batch[i]->k * sizeof(int32_t);
            if (S->in_use + need + b <= S->mem_budget) {
              need += b;
              take.push_back(i);
            } else {
              batch[i]->rows_dropped = 1;
              S->rows_dropped++;
            }
          }
          S->in_use += need;
        }
        if (!take.empty()) {
          const int32_t nr = (int32_t)take.size();
          std::vector<const hm_pattern *> rp(nr);
          std::vector<int32_t> rm(nr);
          std::vector<uint64_t> off2(nr + 1, 0), rc(nr, 0);
          for (int32_t j = 0; j < nr; ++j) {
            const auto &q = batch[take[j]];
            rp[j] = q->pattern;
            rm[j] = q->mode;
            off2[j + 1] = off2[j] + q->count * (uint64_t)q->k;
          }
          int32_t *d2 = nullptr;
          cudaError_t e2 = cudaMallocAsync((void **)&d2, sizeof(int32_t) * std::max<uint64_t>(off2[nr], 1), stream);
          if (e2 != cudaSuccess) {
            (void)cudaGetLastError();
            st = HM_ERR_OOM;
          } else {
            st = hm_enumerate_batch(S->g, rp.data(), rm.data(), nr, d2, off2.data(), rc.data(), stream);
            if (st == HM_OK) {
              for (int32_t j = 0; j < nr; ++j) {
                auto &q = batch[take[j]];
                q->rows.resize(q->count * (uint64_t)q->k);
                if (!q->rows.empty() &&
                    cudaMemcpyAsync(q->rows.data(), d2 + off2[j], sizeof(int32_t) * q->rows.size(),
                                    cudaMemcpyDeviceToHost, stream) != cudaSuccess)
                  st = HM_ERR_CUDA;
              }
              if (cudaStreamSynchronize(stream) != cudaSuccess) st = HM_ERR_CUDA;
            }
            cudaFreeAsync(d2, stream);
          }
        }
        std::lock_guard<std::mutex> lk(S->mu);
        S->in_use -= need;
      }
    }
    const auto t_end = clock_t_::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto &q : batch) {
        q->status = st;
        q->latency_ms = std::chrono::duration<double, std::milli>(t_end - q->t_submit).count();
        q->reserved = 0;
        q->done.store(1);
        S->completed++;
      }
      S->in_use -= held;
      S->inflight_batches--;
    }
    S->cv.notify_all();
    S->done_cv.notify_all();
  }
  cudaStreamSynchronize(stream);
  cudaStreamDestroy(stream);
}

// Arcs per (source label, arc label, target label), from the label-grouped
// directory: each out-directory entry of u is one (arc label, neighbour
// label) group of u's out-arcs.
hm_status label_triples(const hm_graph *g, std::map<std::tuple<int32_t, int32_t, int32_t>, uint64_t> &out) {
  const int32_t n = g->n;
  std::vector<int4> vi(n), vdir(n), dir((size_t)g->ndir_out);
  if (n > 0) {
    HM_CUDA_TRY(cudaMemcpy(vi.data(), g->vi, sizeof(int4) * n, cudaMemcpyDeviceToHost));
    HM_CUDA_TRY(cudaMemcpy(vdir.data(), g->vdir, sizeof(int4) * n, cudaMemcpyDeviceToHost));
  }
  if (g->ndir_out > 0)
    HM_CUDA_TRY(cudaMemcpy(dir.data(), g->gdir_out, sizeof(int4) * (size_t)g->ndir_out, cudaMemcpyDeviceToHost));
  for (int32_t u = 0; u < n; ++u)
    for (int32_t e = vdir[u].x; e < vdir[u].x + vdir[u].y; ++e)
      out[std::make_tuple(vi[u].x, dir[e].x, dir[e].y)] += (uint64_t)(dir[e].w - dir[e].z);
  return HM_OK;
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
  if (cudaSetDevice(g->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete S;
    return HM_ERR_CUDA;
  }
  hm_status st = label_triples(g, S->triples);
  if (st != HM_OK) {
    delete S;
    return st;
  }
  // default: a quarter of the device memory free now, at most 32 GiB
  if (!mem_budget) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      (void)cudaGetLastError();
      free_b = size_t(4) << 30;
    }
    mem_budget = std::min<uint64_t>((uint64_t)free_b / 4, uint64_t(32) << 30);
  }
  S->mem_budget = mem_budget;
  if (S->mem_budget < kBatchFixed) {
    delete S;
    return HM_ERR_ARG;  // the budget cannot admit even one batch
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
  {
    // its depth-2 states: at most the arcs whose labels fit its seeding arc
    const hm::Plan &pl = p->plan[mode];
    const int32_t l0 = pl.vlab[0], l1 = pl.vlab[1];
    const auto key = pl.seed_rev ? std::make_tuple(l1, pl.seed_lab, l0) : std::make_tuple(l0, pl.seed_lab, l1);
    const auto it = S->triples.find(key);
    const uint64_t states = it == S->triples.end() ? 0 : it->second;
    q->need = 2 * 12 * states;  // two seed queues of (int2 state + pattern id)
  }
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
