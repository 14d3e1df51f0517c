// hm_api.cpp -- process-wide settings and small C-ABI helpers.
#include <atomic>

#include "hm_internal.cuh"

namespace hm {
namespace {
std::atomic<uint64_t> g_budget_ms{120000};
std::atomic<uint64_t> g_budget_chunks{0};
std::atomic<int> g_timing{0};
std::atomic<int> g_counters{0};
}  // namespace

hm_stats &tls_stats() {
  static thread_local hm_stats s{};
  return s;
}
bool timing_enabled() { return g_timing.load(std::memory_order_relaxed) != 0; }
bool counters_enabled() { return g_counters.load(std::memory_order_relaxed) != 0; }
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
