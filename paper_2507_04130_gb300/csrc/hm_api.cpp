// hm_api.cpp -- process-wide settings and small C-ABI helpers.
#include <atomic>

#include "hm_internal.cuh"

namespace hm {
namespace {
constexpr int kDefaultFilterMin = 1;
std::atomic<uint64_t> g_budget_ms{120000};
std::atomic<uint64_t> g_budget_chunks{0};
std::atomic<int> g_timing{0};
std::atomic<int> g_counters{0};
std::atomic<int> g_min_blocks{4}, g_split_min{64}, g_pair_mode{0}, g_seeds_per_fetch{1};
std::atomic<int> g_poll_every{128};
std::atomic<int> g_leaf_flatten{1};
std::atomic<int> g_arc_filter{kDefaultFilterMin};
std::atomic<int> g_share_seeds{1};
std::atomic<int> g_symmetry{1};
std::atomic<int> g_warps_per_state{0};  // 0: automatic
std::atomic<int> g_lookahead{-1};
}  // namespace

hm_stats &tls_stats() {
  static thread_local hm_stats s{};
  return s;
}
bool timing_enabled() { return g_timing.load(std::memory_order_relaxed) != 0; }
bool counters_enabled() { return g_counters.load(std::memory_order_relaxed) != 0; }
hm_tuning tuning() {
  hm_tuning t{};
  t.extend_min_blocks = g_min_blocks.load(std::memory_order_relaxed);
  t.split_min = g_split_min.load(std::memory_order_relaxed);
  t.pair_mode = g_pair_mode.load(std::memory_order_relaxed);
  t.seeds_per_fetch = g_seeds_per_fetch.load(std::memory_order_relaxed);
  t.poll_every = g_poll_every.load(std::memory_order_relaxed);
  t.leaf_flatten = g_leaf_flatten.load(std::memory_order_relaxed);
  t.arc_filter = g_arc_filter.load(std::memory_order_relaxed);
  t.share_seeds = g_share_seeds.load(std::memory_order_relaxed);
  t.symmetry = g_symmetry.load(std::memory_order_relaxed);
  t.warps_per_state = g_warps_per_state.load(std::memory_order_relaxed);
  t.lookahead = g_lookahead.load(std::memory_order_relaxed);
  return t;
}
int32_t filter_min() { return g_arc_filter.load(std::memory_order_relaxed); }
uint64_t budget_ms() { return g_budget_ms.load(std::memory_order_relaxed); }
uint64_t budget_chunks() { return g_budget_chunks.load(std::memory_order_relaxed); }
}  // namespace hm

extern "C" const char *hm_status_str(hm_status s) {
  switch (s) {
    case HM_OK: return "ok";
    case HM_ERR_ARG: return "invalid argument";
    case HM_ERR_SELF_LOOP: return "self-loop";
    case HM_ERR_DUP_EDGE: return "duplicate arc";
    case HM_ERR_PATTERN: return "invalid pattern";
    case HM_ERR_OOM: return "out of device memory";
    case HM_ERR_CAPACITY: return "output capacity too small";
    case HM_ERR_BUDGET: return "work budget exhausted";
    case HM_ERR_CUDA: return "CUDA error";
    case HM_ERR_NO_DEVICE: return "no CUDA device";
  }
  return "unknown status";
}

extern "C" hm_status hm_set_budget(uint64_t max_ms, uint64_t max_chunks) {
  hm::g_budget_ms.store(max_ms ? max_ms : 120000);
  hm::g_budget_chunks.store(max_chunks);
  return HM_OK;
}

extern "C" hm_status hm_last_stats(hm_stats *out) {
  if (!out) return HM_ERR_ARG;
  *out = hm::tls_stats();
  return HM_OK;
}

extern "C" hm_status hm_set_timing(int enabled) {
  hm::g_timing.store(enabled ? 1 : 0);
  return HM_OK;
}

extern "C" hm_status hm_set_counters(int enabled) {
  hm::g_counters.store(enabled ? 1 : 0);
  return HM_OK;
}

extern "C" hm_status hm_set_tuning(const hm_tuning *t) {
  if (!t) return HM_ERR_ARG;
  const int mb = t->extend_min_blocks ? t->extend_min_blocks : 4;
  const int sm = t->split_min ? t->split_min : 64;
  const int sp = t->seeds_per_fetch ? t->seeds_per_fetch : 1;
  const int pe = t->poll_every ? t->poll_every : 128;
  if ((mb != 4 && mb != 5 && mb != 6) || sm < 2 || sp < 1 || sp > 1024 ||
      (t->pair_mode != 0 && t->pair_mode != 1) || pe < 1 || pe > 65536 || (pe & (pe - 1)) ||
      t->leaf_flatten < -1 || t->leaf_flatten > 1 || t->arc_filter < -1 || t->share_seeds < -1 ||
      t->share_seeds > 1 || t->symmetry < -1 || t->symmetry > 1 ||
      (t->warps_per_state != 0 && t->warps_per_state != 1 && t->warps_per_state != 2 &&
       t->warps_per_state != 4) ||
      t->lookahead < -1 || t->lookahead > 1)
    return HM_ERR_ARG;
  hm::g_min_blocks.store(mb);
  hm::g_split_min.store(sm);
  hm::g_pair_mode.store(t->pair_mode);
  hm::g_seeds_per_fetch.store(sp);
  hm::g_poll_every.store(pe);
  hm::g_leaf_flatten.store(t->leaf_flatten < 0 ? -1 : 1);
  hm::g_arc_filter.store(t->arc_filter ? t->arc_filter : hm::kDefaultFilterMin);
  hm::g_share_seeds.store(t->share_seeds < 0 ? -1 : 1);
  hm::g_symmetry.store(t->symmetry < 0 ? -1 : 1);
  hm::g_warps_per_state.store(t->warps_per_state);
  hm::g_lookahead.store(t->lookahead > 0 ? 1 : -1);
  return HM_OK;
}

extern "C" hm_status hm_get_tuning(hm_tuning *t) {
  if (!t) return HM_ERR_ARG;
  *t = hm::tuning();
  return HM_OK;
}
