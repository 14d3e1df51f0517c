// hm_match.cu -- single-pattern entry points of the hot path (host orchestration)
// and the count that allocates no device memory.  The kernels they launch are
// in hm_kernels.cuh.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "hm_kernels.cuh"

namespace hm {
namespace {

enum class Want { kCount, kRows, kStates };

// The plan for shared position-0 states: the induced non-arcs between
// position 1 and later positions leave the per-position condition lists and
// become P.defer, read from the chosen image v of position 1.
Plan shared_plan(const Plan &P) {
  Plan Q = P;
  strip_symmetry(Q);  // position 1 is chosen at the leaves; its images are not permuted there
  Q.ndefer = 0;
  for (int p = 2; p < P.k; ++p) {
    int c = 0;
    for (int j = 0; j < P.ncons[p]; ++j) {
      const Cons cs = P.cons[p][j];
      if (cs.q == 1)  // only induced non-arcs can name position 1 here (defer1)
        Q.defer[Q.ndefer++] = Cons{(int8_t)p, cs.kind == kNotOut ? kNotIn : kNotOut, 0, 0};
      else
        Q.cons[p][c++] = cs;
    }
    Q.ncons[p] = c;
  }
  return Q;
}

// Seeds sorted by (u, v): flag the first seed of each position-0 image, and
// (cap > 0) every seed at a multiple of `cap`, so no group holds more than
// cap seeds.  The groups still partition the seeds.
__global__ void k_seed_group_flags(const int2 *__restrict__ s, int64_t n, int64_t cap,
                                   uint32_t *__restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = i < n && (i == 0 || s[i].x != s[i - 1].x || (cap > 0 && i % cap == 0)) ? 1u : 0u;
}

// Seeds per shared group in induced calls: each group's (match, image) pairs
// are checked by its own warp at the leaf, so a hub's hundreds of seeds are
// split into groups of at most this size, which keeps that loop short while
// the search over the later positions still runs about once per 32 seeds
// instead of once per seed.  The cuts fall at every 32nd seed of the whole
// sorted seed list (global alignment), not at every 32nd seed of one image,
// so an image's first and last groups can be smaller: an image with n seeds
// gets at most ceil(n/32) + 1 groups.
constexpr int64_t kInducedGroupCap = 32;

// One int4 {u, first, end, 0} per group; idx is the exclusive scan of flag.
__global__ void k_seed_groups(const int2 *__restrict__ s, int64_t n, const uint32_t *__restrict__ flag,
                              const uint32_t *__restrict__ idx, int4 *__restrict__ groups,
                              unsigned long long *__restrict__ ngroups) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t gi = idx[i] + flag[i] - 1;
    int32_t *gw = reinterpret_cast<int32_t *>(groups + gi);
    if (flag[i]) {
      gw[0] = s[i].x;
      gw[1] = (int32_t)i;
      gw[3] = 0;
    }
    if (i + 1 == n || flag[i + 1]) gw[2] = (int32_t)(i + 1);
    if (i + 1 == n) *ngroups = gi + 1;
  }
}

// First arc of part `part` of `nparts` contiguous CSR ranges (multiple of 4; part == nparts gives m).
int64_t part_start(int64_t m, int32_t part, int32_t nparts) {
  if (part >= nparts) return m;
  return (int64_t)((__int128)m * part / nparts) & ~int64_t(3);
}

hm_status run_match(const hm_graph *g, const hm_pattern *p, hm_mode mode, int32_t root,
                    const uint8_t *root_mask, int32_t *out, uint64_t cap, uint64_t *count,
                    cudaStream_t s, Want want, int32_t part = 0, int32_t nparts = 1) {
  if (!g || !p || !count || (mode != HM_MONO && mode != HM_INDUCED)) return HM_ERR_ARG;
  if (nparts < 1 || part < 0 || part >= nparts) return HM_ERR_ARG;
  if (want != Want::kCount && cap > 0 && !out) return HM_ERR_ARG;
  ensure_pool();
  hm_stats &st = tls_stats();
  std::memset(&st, 0, sizeof(st));
  const bool timing = timing_enabled();
  const bool counters = counters_enabled();
  uint32_t launches = 0;
  Plan plan = p->plan[mode];
  if (root_mask) {
    if (root < 0 || root >= p->k) return HM_ERR_ARG;
    for (int i = 0; i < p->k; ++i)
      if (plan.orig[i] == root) plan.root_pos = i;
    strip_symmetry(plan);  // the root restriction is on one map, not on its orbit
  }
  if (tuning().symmetry < 0) strip_symmetry(plan);
  const DevGraph G = g->dev();
  const int64_t m = g->m;
  Scratch sc(s);
  Ctl *ctl;
  int2 *seeds_a, *seeds_b = nullptr;
  HM_CUDA_TRY(sc.get((void **)&ctl, sizeof(Ctl)));
  HM_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
  HM_CUDA_TRY(sc.get((void **)&seeds_a, sizeof(int2) * (size_t)std::max<int64_t>(m, 1)));
  if (plan.ov_need > 0)
    HM_CUDA_TRY(sc.get((void **)&seeds_b, sizeof(int2) * (size_t)std::max<int64_t>(m, 1)));
  const int sms = num_sms();

  // a2 + a3: edge scan with the vertex and edge validators
  Timer t_edge(s, timing);
  const int64_t e_begin = part_start(m, part, nparts), e_end = part_start(m, part + 1, nparts);
  {
    NvtxRange r_edge("hm.edge_scan");
    int64_t groups = (e_end - e_begin + 3) / 4;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>((groups + kSeedThreads - 1) / kSeedThreads,
                                                           (int64_t)sms * 8));
    if (e_end > e_begin) {
      if (counters)
        k_edge_seed<true><<<grid, kSeedThreads, 0, s>>>(G, plan, root_mask, seeds_a, (unsigned long long)m,
                                                        &ctl->nseeds_raw, &ctl->bytes_edge, e_begin, e_end);
      else
        k_edge_seed<false><<<grid, kSeedThreads, 0, s>>>(G, plan, root_mask, seeds_a, (unsigned long long)m,
                                                         &ctl->nseeds_raw, &ctl->bytes_edge, e_begin, e_end);
      ++launches;
    }
    t_edge.stop();
    HM_CUDA_TRY(cudaGetLastError());
  }
  const int2 *seeds = seeds_a;
  const unsigned long long *nseeds = &ctl->nseeds_raw;
  Timer t_ov(s, timing && plan.ov_need > 0);
  if (plan.ov_need > 0) {
    NvtxRange r_ov("hm.overlap_test");
    if (counters)
      k_seed_overlap<true><<<sms * 8, kSeedThreads, 0, s>>>(G, plan.ov_need, seeds_a, &ctl->nseeds_raw,
                                                            seeds_b, (unsigned long long)m, &ctl->nseeds,
                                                            &ctl->bytes_overlap);
    else
      k_seed_overlap<false><<<sms * 8, kSeedThreads, 0, s>>>(G, plan.ov_need, seeds_a, &ctl->nseeds_raw,
                                                             seeds_b, (unsigned long long)m, &ctl->nseeds,
                                                             &ctl->bytes_overlap);
    ++launches;
    t_ov.stop();
    HM_CUDA_TRY(cudaGetLastError());
    seeds = seeds_b;
    nseeds = &ctl->nseeds;
  }

  if (want == Want::kStates) {
    Ctl h;
    HM_CUDA_TRY(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    HM_CUDA_TRY(cudaStreamSynchronize(s));
    unsigned long long n = plan.ov_need > 0 ? h.nseeds : h.nseeds_raw;
    *count = n;
    if (n > cap) return HM_ERR_CAPACITY;
    if (n)
      HM_CUDA_TRY(cudaMemcpyAsync(out, seeds, sizeof(int2) * n, cudaMemcpyDeviceToDevice, s));
    return HM_OK;
  }

  // Shared position-0 states: group the seeds by their position-0 image
  // (induced calls: at most kInducedGroupCap seeds per group).
  const hm_tuning tu = tuning();
  const bool share = p->k > 2 && plan.defer1 && tu.share_seeds > 0;
  const int4 *groups = nullptr;
  Timer t_grp(s, timing && share);
  if (share) {
    NvtxRange r_grp("hm.group_seeds");
    unsigned long long ns = 0;
    HM_CUDA_TRY(cudaMemcpyAsync(&ns, nseeds, sizeof(ns), cudaMemcpyDeviceToHost, s));
    HM_CUDA_TRY(cudaStreamSynchronize(s));
    int32_t *tmp;
    uint32_t *flag, *idx;
    int4 *gr;
    HM_CUDA_TRY(sc.get((void **)&tmp, sizeof(int2) * (size_t)std::max<unsigned long long>(ns, 1)));
    HM_CUDA_TRY(sc.get((void **)&flag, sizeof(uint32_t) * (size_t)(ns + 1)));
    HM_CUDA_TRY(sc.get((void **)&idx, sizeof(uint32_t) * (size_t)(ns + 1)));
    HM_CUDA_TRY(sc.get((void **)&gr, sizeof(int4) * (size_t)std::max<unsigned long long>(ns, 1)));
    HM_CUDA_TRY(cudaMemsetAsync(&ctl->ngroups, 0, sizeof(unsigned long long), s));
    if (ns > 0) {
      const int cols[2] = {0, 1};
      int2 *sd = const_cast<int2 *>(seeds);
      int nl = 0;
      hm_status r = radix_sort_rows(reinterpret_cast<int32_t *>(sd), tmp, (int64_t)ns, 2, cols, 2,
                                    bits_for(g->n), s, &nl);
      if (r != HM_OK) return r;
      launches += nl;
      const int gb = (int)std::min<unsigned long long>((ns + 256) / 256, (unsigned long long)sms * 8);
      k_seed_group_flags<<<gb, 256, 0, s>>>(seeds, (int64_t)ns, plan.induced ? kInducedGroupCap : 0, flag);
      r = exclusive_scan_u32(flag, idx, (int64_t)ns + 1, s);
      if (r != HM_OK) return r;
      k_seed_groups<<<gb, 256, 0, s>>>(seeds, (int64_t)ns, flag, idx, gr, &ctl->ngroups);
      launches += 5;
      HM_CUDA_TRY(cudaGetLastError());
    }
    groups = gr;
    plan = shared_plan(plan);
  }
  t_grp.stop();

  // a4 + a5: state injection and extension
  const bool rows = want == Want::kRows;
  Timer t_ext(s, timing && p->k > 2);
  {  // the extension's launches
  NvtxRange r_ext("hm.extend");
  if (p->k == 2) {
    k_seed_rows<<<sms * 4, 256, 0, s>>>(plan, seeds, nseeds, rows ? out : nullptr, cap, ctl);
    ++launches;
    HM_CUDA_TRY(cudaGetLastError());
  } else {
    Task *qbuf;
    unsigned long long *qseq;
    HM_CUDA_TRY(sc.get((void **)&qbuf, sizeof(Task) * kQueueCap));
    HM_CUDA_TRY(sc.get((void **)&qseq, sizeof(unsigned long long) * kQueueCap));
    k_qinit<<<64, 256, 0, s>>>(qseq);
    ++launches;
    ExtArgs A{};
    A.seeds = seeds;
    A.nseeds = nseeds;
    if (share) {
      A.groups = groups;
      A.sorted_seeds = seeds;
      A.nseeds = &ctl->ngroups;
    }
    A.qbuf = qbuf;
    A.qseq = qseq;
    A.ctl = ctl;
    A.rows = rows ? out : nullptr;
    A.cap = rows ? cap : 0;
    A.root_mask = root_mask;
    A.budget_ns = budget_ms() * 1000000ull;
    A.max_chunks = budget_chunks();
    A.split_min = tu.split_min;
    A.pair_mode = tu.pair_mode;
    A.seeds_per_fetch = tu.seeds_per_fetch;
    A.poll_mask = (uint32_t)tu.poll_every - 1u;
    A.leaf_flatten = tu.leaf_flatten > 0 ? 1 : 0;
    A.wps_shift = wps_shift(tu, share);
    A.lookahead = tu.lookahead > 0 ? 1 : 0;
    const int slot = min_blocks_slot(tu.extend_min_blocks);
    const size_t smem = warp_smem_bytes(plan.ngrp) * kExtWarps;
    const bool sym = plan.naut > 1;
    const int grid = extend_grid(rows, counters, smem, slot, share, sym);
    if (grid <= 0) return HM_ERR_CUDA;
    st.extend_grid = grid;
    st.extend_block = kExtThreads;
    extend_kernel(rows, counters, slot, share, sym)<<<grid, kExtThreads, smem, s>>>(G, plan, A);
    ++launches;
    t_ext.stop();
    HM_CUDA_TRY(cudaGetLastError());
  }
  }
  Ctl h;
  HM_CUDA_TRY(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  HM_CUDA_TRY(cudaStreamSynchronize(s));
  st.ms_edge_scan = t_edge.ms();
  st.ms_overlap = t_ov.ms() + t_grp.ms();
  st.ms_extend = t_ext.ms();
  st.seeds_scanned = (uint64_t)(e_end - e_begin);
  st.states_injected = plan.ov_need > 0 ? h.nseeds : h.nseeds_raw;
  st.tasks_donated = h.donated;
  st.chunks = h.chunks;
  st.matches = h.count;
  st.bytes_edge_scan = h.bytes_edge;
  st.bytes_overlap = h.bytes_overlap;
  st.bytes_extend = h.bytes_extend;
  st.model_bytes_edge_scan = h.bytes_edge_model;
  st.model_bytes_overlap = h.bytes_overlap_model;
  st.model_bytes_extend = h.bytes_extend_model;
  st.candidates = h.lanes;
  for (int i = 0; i < kMaxK; ++i) {
    st.level_chunks[i] = h.level_chunks[i];
    st.level_candidates[i] = h.level_lanes[i];
  }
  st.kernel_launches = launches;
  if (h.status == kStatBudget) return HM_ERR_BUDGET;
  if (h.status != kStatOk) return HM_ERR_CUDA;
  *count = h.count;
  if (!rows) return HM_OK;
  if (h.count > cap) return HM_ERR_CAPACITY;
  if (h.count > 1) {
    NvtxRange r_sort("hm.sort_rows");
    Timer t(s, timing);
    int32_t *tmp;
    HM_CUDA_TRY(sc.get((void **)&tmp, sizeof(int32_t) * (size_t)h.count * p->k));
    int cols[kMaxK];
    for (int i = 0; i < p->k; ++i) cols[i] = i;
    const int sort_cols = p->k;
    int nl = 0;
    hm_status r = radix_sort_rows(out, tmp, (int64_t)h.count, p->k, cols, sort_cols, bits_for(g->n), s, &nl);
    st.kernel_launches += nl;
    t.stop();
    if (r != HM_OK) return r;
    if (timing) {
      HM_CUDA_TRY(cudaStreamSynchronize(s));
      st.ms_sort = t.ms();
    }
  }
  return HM_OK;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" hm_status hm_count_matches(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                      uint64_t *count, void *stream) {
  return run_match(g, p, mode, -1, nullptr, nullptr, 0, count, (cudaStream_t)stream, Want::kCount);
}

extern "C" hm_status hm_enumerate_matches(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                          int32_t *rows_dev, uint64_t cap, uint64_t *count,
                                          void *stream) {
  return run_match(g, p, mode, -1, nullptr, rows_dev, cap, count, (cudaStream_t)stream, Want::kRows);
}

extern "C" hm_status hm_count_matches_rooted(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                             int32_t root, const uint8_t *root_mask_dev,
                                             uint64_t *count, void *stream) {
  if (!root_mask_dev) return HM_ERR_ARG;
  return run_match(g, p, mode, root, root_mask_dev, nullptr, 0, count, (cudaStream_t)stream,
                   Want::kCount);
}

extern "C" hm_status hm_count_matches_part(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                           int32_t part, int32_t nparts, uint64_t *count,
                                           void *stream) {
  return run_match(g, p, mode, -1, nullptr, nullptr, 0, count, (cudaStream_t)stream, Want::kCount,
                   part, nparts);
}

extern "C" hm_status hm_enumerate_matches_part(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                               int32_t part, int32_t nparts, int32_t *rows_dev,
                                               uint64_t cap, uint64_t *count, void *stream) {
  return run_match(g, p, mode, -1, nullptr, rows_dev, cap, count, (cudaStream_t)stream, Want::kRows,
                   part, nparts);
}

extern "C" hm_status hm_injected_states(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                        int32_t *states_dev, uint64_t cap, uint64_t *count,
                                        void *stream) {
  return run_match(g, p, mode, -1, nullptr, states_dev, cap, count, (cudaStream_t)stream,
                   Want::kStates);
}

// ---------------------------------------------------------------------------
// Counting without any device allocation (hm_count_matches_static).
// It runs one search per depth-2 state: grouping the states by their
// position-0 image (share_seeds) sorts them into temporary buffers that the
// fixed array has no room for.
//
// Some callers cannot allocate device memory while they match: a process
// whose device memory is carved up in advance by another allocator (a
// framework's caching pool, or a hard per-process budget) and must not take
// more, or a latency-critical loop where a cudaMalloc, which may synchronise
// the whole device, is not acceptable.  For them this entry point takes every
// byte of working memory -- the control block, the donation queue and the two
// seed queues -- from one file-scope device array of fixed size.  Every GPU
// that loads the library holds that array until the process exits; every call
// on a device shares it, so calls whose work overlaps on the GPU (for example
// on two streams) race on it and must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace hm {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr size_t kStaticCtlBytes = 4096;  // fixed room for the control block
static_assert(sizeof(Ctl) <= kStaticCtlBytes, "control block outgrew its static room");
constexpr size_t kStaticQseqBytes = sizeof(unsigned long long) * kQueueCap;
constexpr size_t kStaticQbufBytes = sizeof(Task) * kQueueCap;
constexpr size_t kStaticSeedBase = kStaticCtlBytes + kStaticQseqBytes + kStaticQbufBytes;
// two seed queues of int2, each able to hold one state per target arc
constexpr int64_t kStaticMaxArcs =
    (int64_t)((kStaticScratchBytes - kStaticSeedBase) / (2 * sizeof(int2)));
static_assert(kStaticSeedBase % 256 == 0, "static scratch layout alignment");
static_assert(kStaticMaxArcs == HM_STATIC_MAX_ARCS, "header constant out of date");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_lock;
void *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
hm_status static_scratch(void **out) {
  int dev = 0;
  HM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return HM_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_static_lock);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return HM_ERR_CUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return HM_OK;
}

}  // namespace
}  // namespace hm

extern "C" hm_status hm_count_matches_static(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                             uint64_t *count, void *stream) {
  using namespace hm;
  if (!g || !p || !count || (mode != HM_MONO && mode != HM_INDUCED)) return HM_ERR_ARG;
  if (g->m > kStaticMaxArcs) return HM_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  void *base = nullptr;
  hm_status rc = static_scratch(&base);
  if (rc != HM_OK) return rc;
  unsigned char *b = static_cast<unsigned char *>(base);
  Ctl *ctl = reinterpret_cast<Ctl *>(b);
  unsigned long long *qseq = reinterpret_cast<unsigned long long *>(b + kStaticCtlBytes);
  Task *qbuf = reinterpret_cast<Task *>(b + kStaticCtlBytes + kStaticQseqBytes);
  int2 *seeds_a = reinterpret_cast<int2 *>(b + kStaticSeedBase);
  int2 *seeds_b = seeds_a + kStaticMaxArcs;

  hm_stats &st = tls_stats();
  std::memset(&st, 0, sizeof(st));
  Plan plan = p->plan[mode];
  if (tuning().symmetry < 0) strip_symmetry(plan);
  const DevGraph G = g->dev();
  const int64_t m = g->m;
  const int sms = num_sms();
  uint32_t launches = 0;
  // the array keeps the previous call's contents: clear the control block and the queue
  HM_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
  k_qinit<<<64, 256, 0, s>>>(qseq);
  ++launches;
  if (m) {
    const int64_t groups = (m + 3) / 4;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((groups + kSeedThreads - 1) / kSeedThreads, (int64_t)sms * 8));
    k_edge_seed<false><<<grid, kSeedThreads, 0, s>>>(G, plan, nullptr, seeds_a,
                                                     (unsigned long long)kStaticMaxArcs,
                                                     &ctl->nseeds_raw, &ctl->bytes_edge, 0, m);
    ++launches;
  }
  const int2 *seeds = seeds_a;
  const unsigned long long *nseeds = &ctl->nseeds_raw;
  if (plan.ov_need > 0) {
    k_seed_overlap<false><<<sms * 8, kSeedThreads, 0, s>>>(
        G, plan.ov_need, seeds_a, &ctl->nseeds_raw, seeds_b, (unsigned long long)kStaticMaxArcs,
        &ctl->nseeds, &ctl->bytes_overlap);
    ++launches;
    seeds = seeds_b;
    nseeds = &ctl->nseeds;
  }
  if (p->k == 2) {
    k_seed_rows<<<sms * 4, 256, 0, s>>>(plan, seeds, nseeds, nullptr, 0, ctl);
    ++launches;
  } else {
    ExtArgs A{};
    A.seeds = seeds;
    A.nseeds = nseeds;
    A.qbuf = qbuf;
    A.qseq = qseq;
    A.ctl = ctl;
    A.rows = nullptr;
    A.cap = 0;
    A.root_mask = nullptr;
    A.budget_ns = budget_ms() * 1000000ull;
    A.max_chunks = budget_chunks();
    const hm_tuning tu = tuning();
    A.split_min = tu.split_min;
    A.pair_mode = tu.pair_mode;
    A.seeds_per_fetch = tu.seeds_per_fetch;
    A.poll_mask = (uint32_t)tu.poll_every - 1u;
    A.leaf_flatten = tu.leaf_flatten > 0 ? 1 : 0;
    A.wps_shift = wps_shift(tu);
    A.lookahead = tu.lookahead > 0 ? 1 : 0;
    const int slot = min_blocks_slot(tu.extend_min_blocks);
    const size_t smem = warp_smem_bytes(plan.ngrp) * kExtWarps;
    const bool sym = plan.naut > 1;
    const int grid = extend_grid(false, false, smem, slot, false, sym);
    if (grid <= 0) return HM_ERR_CUDA;
    extend_kernel(false, false, slot, false, sym)<<<grid, kExtThreads, smem, s>>>(G, plan, A);
    ++launches;
  }
  HM_CUDA_TRY(cudaGetLastError());
  Ctl h;
  HM_CUDA_TRY(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  HM_CUDA_TRY(cudaStreamSynchronize(s));
  st.seeds_scanned = (uint64_t)m;
  st.states_injected = plan.ov_need > 0 ? h.nseeds : h.nseeds_raw;
  st.tasks_donated = h.donated;
  st.chunks = h.chunks;
  st.matches = h.count;
  st.kernel_launches = launches;
  if (h.status == kStatBudget) return HM_ERR_BUDGET;
  if (h.status != kStatOk) return HM_ERR_CUDA;
  *count = h.count;
  return HM_OK;
}
