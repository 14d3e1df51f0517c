// hm_batch.cu -- many patterns against one resident graph in one pass.
//
// The HiPerMotif algorithm (Sec. III-C) runs one edge loop per pattern.  A
// batch shares that loop: one scan of the target's arcs tries every arc as
// the seeding arc of every pattern whose signature (arc label, label of the
// arc's source, label of its target) it carries -- looked up in a small hash
// table built on the host -- and applies that pattern's vertex and edge
// validators (Alg. 2, Alg. 3).  Survivors carry their pattern id through the
// overlap test and into ONE persistent extension launch, whose warps take
// depth-2 states of any pattern and read the pattern's plan from a device
// table.  Rows of all patterns are sorted in one stable radix sort keyed on
// (pattern id, row), then written back to each pattern's region.
#include <algorithm>
#include <cstring>
#include <vector>

#include "hm_kernels.cuh"

namespace hm {
namespace {

// seeding-arc signature table (open addressing, linear probing)
struct SigKey {
  int32_t lab, vsrc, vdst, used;
};

__device__ __host__ __forceinline__ uint32_t sig_hash(int32_t lab, int32_t vs, int32_t vd) {
  uint32_t h = (uint32_t)lab * 0x9E3779B1u;
  h ^= (uint32_t)vs + 0x7F4A7C15u + (h << 6) + (h >> 2);
  h ^= (uint32_t)vd + 0x94D049BBu + (h << 6) + (h >> 2);
  return h;
}

struct SigTable {
  const SigKey *keys;
  const int2 *vals;       // {first, count} into pids
  const int32_t *pids;    // patterns sharing a signature
  uint32_t mask;
};

// The batch's seed test for one (arc, pattern) pair: Alg. 2 on the position-0
// image and Alg. 3's label, opposite-arc and degree checks, with the seeding
// direction of that pattern.
__device__ __forceinline__ bool seed_test_batch(const DevGraph &G, const Plan &P, int32_t a,
                                                int32_t b, int4 ia, int4 ib, int2 *out) {
  const int32_t u = P.seed_rev ? b : a;
  const int32_t v = P.seed_rev ? a : b;
  const int4 iu = P.seed_rev ? ib : ia;
  const int4 iv = P.seed_rev ? ia : ib;
  if (iu.y < P.dout[0] || iu.z < P.din[0]) return false;
  if (iv.y < P.dout[1] || iv.z < P.din[1]) return false;
  if (P.back_req | P.back_forbid) {
    int32_t lab = 0;
    Bytes unused;
    const bool found = arc_lookup<false>(G, b, a, ib.y, ia.z, &lab, unused);
    if (P.back_req && (!found || lab != P.back_lab)) return false;
    if (P.back_forbid && found) return false;
  }
  *out = make_int2(u, v);
  return true;
}

// Pass 1 (kWrite = false) counts the (arc, pattern) survivors; pass 2 writes
// them.  One atomic per warp and round reserves the warp's output slots.
template <bool kWrite>
__global__ void __launch_bounds__(kSeedThreads)
k_edge_seed_batch(const __grid_constant__ DevGraph G, const Plan *__restrict__ plans,
                  const __grid_constant__ SigTable T, int2 *__restrict__ seeds,
                  int32_t *__restrict__ seed_pid, unsigned long long cap,
                  unsigned long long *__restrict__ nseeds) {
  const int lane = threadIdx.x & 31;
  for (int64_t e0 = (int64_t)blockIdx.x * kSeedThreads; e0 < G.m;
       e0 += (int64_t)gridDim.x * kSeedThreads) {
    const int64_t e = e0 + threadIdx.x;
    int32_t first = 0, cnt = 0, a = 0, b = 0;
    int4 ia = make_int4(0, 0, 0, 0), ib = ia;
    if (e < G.m) {
      a = __ldg(G.src + HM_AT(G, e, G.m, kChkList));
      b = __ldg(G.out_adj + HM_AT(G, e, G.m, kChkList));
      const int32_t l = __ldg(G.out_elab + HM_AT(G, e, G.m, kChkList));
      ia = __ldg(&G.vi[HM_AT(G, a, G.n, kChkVertex)]);
      ib = __ldg(&G.vi[HM_AT(G, b, G.n, kChkVertex)]);
      uint32_t h = sig_hash(l, ia.x, ib.x) & T.mask;
      for (uint32_t probe = 0; probe <= T.mask; ++probe, h = (h + 1) & T.mask) {
        const SigKey k = T.keys[h];
        if (!k.used) break;
        if (k.lab == l && k.vsrc == ia.x && k.vdst == ib.x) {
          const int2 r = T.vals[h];
          first = r.x;
          cnt = r.y;
          break;
        }
      }
    }
    // count this arc's survivors, then reserve slots warp-wide
    uint32_t mine = 0;
    for (int32_t i = 0; i < cnt; ++i) {
      int2 uv;
      mine += seed_test_batch(G, plans[T.pids[first + i]], a, b, ia, ib, &uv);
    }
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(nseeds, (unsigned long long)total);
    base = __shfl_sync(kFull, base, 31);
    if (kWrite && mine) {
      unsigned long long at = base + incl - mine;
      for (int32_t i = 0; i < cnt; ++i) {
        const int32_t pid = T.pids[first + i];
        int2 uv;
        if (seed_test_batch(G, plans[pid], a, b, ia, ib, &uv)) {
          if (at < cap) {
            seeds[at] = uv;
            seed_pid[at] = pid;
          }
          ++at;
        }
      }
    }
  }
}

// Before the overlap test: seeds of patterns without one go straight to the
// output (out / nout); the others are gathered for the test (test / ntest).
// One thread per seed, warp-aggregated appends, so the warp-per-seed test
// runs only where a pattern asks for it.
__global__ void __launch_bounds__(kSeedThreads)
k_overlap_split(const Plan *__restrict__ plans, const int2 *__restrict__ in, const int32_t *__restrict__ pid_in,
                const unsigned long long *__restrict__ nin, int2 *__restrict__ out, int32_t *__restrict__ pid_out,
                unsigned long long *__restrict__ nout, int2 *__restrict__ test, int32_t *__restrict__ pid_test,
                unsigned long long *__restrict__ ntest) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const unsigned long long n = *nin;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n;
       base += stride) {
    const unsigned long long i = base + lane;
    const bool valid = i < n;
    const int32_t pid = valid ? pid_in[i] : 0;
    const int2 uv = valid ? in[i] : make_int2(0, 0);
    const bool pass = valid && plans[pid].ov_need == 0;
    const bool tst = valid && !pass;
    const uint32_t bp = __ballot_sync(kFull, pass), bt = __ballot_sync(kFull, tst);
    unsigned long long op = 0, ot = 0;
    if (lane == 0) {
      if (bp) op = atomicAdd(nout, (unsigned long long)__popc(bp));
      if (bt) ot = atomicAdd(ntest, (unsigned long long)__popc(bt));
    }
    op = __shfl_sync(kFull, op, 0);
    ot = __shfl_sync(kFull, ot, 0);
    if (pass) {
      const unsigned long long at = op + __popc(bp & lt);
      out[at] = uv;
      pid_out[at] = pid;
    }
    if (tst) {
      const unsigned long long at = ot + __popc(bt & lt);
      test[at] = uv;
      pid_test[at] = pid;
    }
  }
}

// Rows of every pattern, padded to width kmax+1 with the pattern id first.
__global__ void k_pack_rows(const int32_t *__restrict__ rows, const unsigned long long *__restrict__ off,
                            const unsigned long long *__restrict__ start, const int32_t *__restrict__ ks,
                            int32_t npat, unsigned long long total, int width,
                            int32_t *__restrict__ packed) {
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < total;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = npat - 1;  // last pattern whose start <= t
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int32_t p = lo, k = ks[p];
    const int32_t *src = rows + off[p] + (t - start[p]) * k;
    int32_t *dst = packed + t * width;
    dst[0] = p;
    for (int c = 0; c < width - 1; ++c) dst[1 + c] = c < k ? src[c] : 0;
  }
}

__global__ void k_unpack_rows(const int32_t *__restrict__ packed, const unsigned long long *__restrict__ off,
                              const unsigned long long *__restrict__ start, const int32_t *__restrict__ ks,
                              unsigned long long total, int width, int32_t *__restrict__ rows) {
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < total;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const int32_t *src = packed + t * width;
    const int32_t p = src[0], k = ks[p];
    int32_t *dst = rows + off[p] + (t - start[p]) * k;
    for (int c = 0; c < k; ++c) dst[c] = src[1 + c];
  }
}

// fit (may be NULL): instead of failing with HM_ERR_CAPACITY when some
// pattern's rows exceed its region, return every count, sort the rows of the
// patterns that fit and flag them (fit[i] = 1); the others' rows are not valid.
hm_status run_batch(const hm_graph *g, const hm_pattern *const *pats, const int32_t *modes,
                    int32_t npat, int32_t *rows, const uint64_t *row_offsets, uint64_t *counts,
                    cudaStream_t s, uint8_t *fit = nullptr) {
  if (!g || npat < 0 || (npat > 0 && (!pats || !modes || !counts))) return HM_ERR_ARG;
  if (npat == 0) return HM_OK;
  const bool want_rows = rows != nullptr || row_offsets != nullptr;
  if (want_rows && (!rows || !row_offsets)) return HM_ERR_ARG;
  ensure_pool();
  hm_stats &st = tls_stats();
  std::memset(&st, 0, sizeof(st));
  const bool timing = timing_enabled();

  // ---- host tables: plans, signatures, row regions
  std::vector<Plan> plans(npat);
  std::vector<int32_t> ks(npat);
  int32_t grp_slots = 0, kmax = 0;
  for (int32_t i = 0; i < npat; ++i) {
    if (!pats[i] || (modes[i] != HM_MONO && modes[i] != HM_INDUCED)) return HM_ERR_ARG;
    plans[i] = pats[i]->plan[modes[i]];
    if (tuning().symmetry < 0) strip_symmetry(plans[i]);
    ks[i] = pats[i]->k;
    grp_slots = std::max(grp_slots, plans[i].ngrp);
    kmax = std::max(kmax, ks[i]);
  }
  std::vector<unsigned long long> off(npat + 1, 0), cap(npat, 0);
  if (want_rows) {
    for (int32_t i = 0; i < npat; ++i) {
      if (row_offsets[i + 1] < row_offsets[i]) return HM_ERR_ARG;
      off[i] = row_offsets[i];
      cap[i] = (row_offsets[i + 1] - row_offsets[i]) / (uint64_t)ks[i];
    }
  }
  // signature (arc label, label of the arc's source, label of its target) -> patterns
  struct Sig {
    int32_t lab, vs, vd, pid;
  };
  std::vector<Sig> sigs(npat);
  for (int32_t i = 0; i < npat; ++i) {
    const Plan &P = plans[i];
    // normal seeding: arc (f(0), f(1)); reversed: arc (f(1), f(0))
    sigs[i] = P.seed_rev ? Sig{P.seed_lab, P.vlab[1], P.vlab[0], i} : Sig{P.seed_lab, P.vlab[0], P.vlab[1], i};
  }
  std::sort(sigs.begin(), sigs.end(), [](const Sig &x, const Sig &y) {
    if (x.lab != y.lab) return x.lab < y.lab;
    if (x.vs != y.vs) return x.vs < y.vs;
    if (x.vd != y.vd) return x.vd < y.vd;
    return x.pid < y.pid;
  });
  uint32_t tsize = 16;
  while (tsize < 2u * (uint32_t)npat) tsize <<= 1;
  std::vector<SigKey> keys(tsize, SigKey{0, 0, 0, 0});
  std::vector<int2> vals(tsize, make_int2(0, 0));
  std::vector<int32_t> pid_list(npat);
  for (int32_t i = 0; i < npat;) {
    int32_t j = i;
    while (j < npat && sigs[j].lab == sigs[i].lab && sigs[j].vs == sigs[i].vs && sigs[j].vd == sigs[i].vd) {
      pid_list[j] = sigs[j].pid;
      ++j;
    }
    uint32_t h = sig_hash(sigs[i].lab, sigs[i].vs, sigs[i].vd) & (tsize - 1);
    while (keys[h].used) h = (h + 1) & (tsize - 1);
    keys[h] = SigKey{sigs[i].lab, sigs[i].vs, sigs[i].vd, 1};
    vals[h] = make_int2(i, j - i);
    i = j;
  }

  // ---- device copies
  Scratch sc(s);
  Plan *d_plans;
  SigKey *d_keys;
  int2 *d_vals;
  int32_t *d_pids, *d_ks;
  unsigned long long *d_ull;  // counts, off, cap, cursor, start, nseeds x2
  Ctl *ctl;
  HM_CUDA_TRY(sc.get((void **)&d_plans, sizeof(Plan) * npat));
  HM_CUDA_TRY(sc.get((void **)&d_keys, sizeof(SigKey) * tsize));
  HM_CUDA_TRY(sc.get((void **)&d_vals, sizeof(int2) * tsize));
  HM_CUDA_TRY(sc.get((void **)&d_pids, sizeof(int32_t) * npat));
  HM_CUDA_TRY(sc.get((void **)&d_ks, sizeof(int32_t) * npat));
  HM_CUDA_TRY(sc.get((void **)&d_ull, sizeof(unsigned long long) * (size_t)(5 * npat + 2)));
  HM_CUDA_TRY(sc.get((void **)&ctl, sizeof(Ctl)));
  unsigned long long *d_counts = d_ull, *d_off = d_ull + npat, *d_cap = d_ull + 2 * npat,
                     *d_cursor = d_ull + 3 * npat, *d_start = d_ull + 4 * npat;
  HM_CUDA_TRY(cudaMemcpyAsync(d_plans, plans.data(), sizeof(Plan) * npat, cudaMemcpyHostToDevice, s));
  HM_CUDA_TRY(cudaMemcpyAsync(d_keys, keys.data(), sizeof(SigKey) * tsize, cudaMemcpyHostToDevice, s));
  HM_CUDA_TRY(cudaMemcpyAsync(d_vals, vals.data(), sizeof(int2) * tsize, cudaMemcpyHostToDevice, s));
  HM_CUDA_TRY(cudaMemcpyAsync(d_pids, pid_list.data(), sizeof(int32_t) * npat, cudaMemcpyHostToDevice, s));
  HM_CUDA_TRY(cudaMemcpyAsync(d_ks, ks.data(), sizeof(int32_t) * npat, cudaMemcpyHostToDevice, s));
  HM_CUDA_TRY(cudaMemsetAsync(d_ull, 0, sizeof(unsigned long long) * (size_t)(5 * npat + 2), s));
  HM_CUDA_TRY(cudaMemcpyAsync(d_off, off.data(), sizeof(unsigned long long) * npat, cudaMemcpyHostToDevice, s));
  HM_CUDA_TRY(cudaMemcpyAsync(d_cap, cap.data(), sizeof(unsigned long long) * npat, cudaMemcpyHostToDevice, s));
  HM_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
  const SigTable T{d_keys, d_vals, d_pids, tsize - 1};
  const DevGraph G = g->dev();
  const int64_t m = g->m;
  const int sms = num_sms();
  uint32_t launches = 0;

  // ---- edge scan: count, size, write
  NvtxRange r_edge("hm.batch_edge_scan");
  Timer t_edge(s, timing);
  const int grid_e = (int)std::max<int64_t>(1, std::min<int64_t>((m + kSeedThreads - 1) / kSeedThreads,
                                                                   (int64_t)sms * 8));
  unsigned long long nraw = 0;
  if (m) {
    k_edge_seed_batch<false><<<grid_e, kSeedThreads, 0, s>>>(G, d_plans, T, nullptr, nullptr, 0,
                                                             &ctl->nseeds_raw);
    HM_CUDA_TRY(cudaMemcpyAsync(&nraw, &ctl->nseeds_raw, sizeof(nraw), cudaMemcpyDeviceToHost, s));
    HM_CUDA_TRY(cudaStreamSynchronize(s));
    launches += 1;
  }
  int2 *seeds_a, *seeds_b;
  int32_t *pid_a, *pid_b;
  HM_CUDA_TRY(sc.get((void **)&seeds_a, sizeof(int2) * (size_t)std::max<unsigned long long>(nraw, 1)));
  HM_CUDA_TRY(sc.get((void **)&pid_a, sizeof(int32_t) * (size_t)std::max<unsigned long long>(nraw, 1)));
  HM_CUDA_TRY(sc.get((void **)&seeds_b, sizeof(int2) * (size_t)std::max<unsigned long long>(nraw, 1)));
  HM_CUDA_TRY(sc.get((void **)&pid_b, sizeof(int32_t) * (size_t)std::max<unsigned long long>(nraw, 1)));
  if (nraw) {
    HM_CUDA_TRY(cudaMemsetAsync(&ctl->nseeds_raw, 0, sizeof(unsigned long long), s));
    k_edge_seed_batch<true><<<grid_e, kSeedThreads, 0, s>>>(G, d_plans, T, seeds_a, pid_a, nraw,
                                                            &ctl->nseeds_raw);
    launches += 1;
  }
  t_edge.stop();
  HM_CUDA_TRY(cudaGetLastError());
  // ---- overlap test (patterns without one pass their seeds through)
  bool any_ov = false;
  for (const Plan &P : plans) any_ov |= P.ov_need > 0;
  const int2 *seeds = seeds_a;
  const int32_t *seed_pid = pid_a;
  const unsigned long long *nseeds = &ctl->nseeds_raw;
  Timer t_ov(s, timing && any_ov);
  if (any_ov && nraw) {
    int2 *seeds_c;
    int32_t *pid_c;
    unsigned long long *ntest;
    HM_CUDA_TRY(sc.get((void **)&seeds_c, sizeof(int2) * (size_t)nraw));
    HM_CUDA_TRY(sc.get((void **)&pid_c, sizeof(int32_t) * (size_t)nraw));
    HM_CUDA_TRY(sc.get((void **)&ntest, sizeof(unsigned long long)));
    HM_CUDA_TRY(cudaMemsetAsync(ntest, 0, sizeof(unsigned long long), s));
    const int grid_s = (int)std::max<unsigned long long>(
        1, std::min<unsigned long long>((nraw + kSeedThreads - 1) / kSeedThreads, (unsigned long long)sms * 8));
    k_overlap_split<<<grid_s, kSeedThreads, 0, s>>>(d_plans, seeds_a, pid_a, &ctl->nseeds_raw, seeds_b, pid_b,
                                                     &ctl->nseeds, seeds_c, pid_c, ntest);
    k_seed_overlap<false, true><<<sms * 8, kSeedThreads, 0, s>>>(G, 0, seeds_c, ntest, seeds_b, nraw,
                                                                  &ctl->nseeds, &ctl->bytes_overlap, d_plans,
                                                                  pid_c, pid_b);
    launches += 2;
    seeds = seeds_b;
    seed_pid = pid_b;
    nseeds = &ctl->nseeds;
  }
  t_ov.stop();

  // ---- one persistent extension launch for every pattern
  Task *qbuf;
  unsigned long long *qseq;
  HM_CUDA_TRY(sc.get((void **)&qbuf, sizeof(Task) * kQueueCap));
  HM_CUDA_TRY(sc.get((void **)&qseq, sizeof(unsigned long long) * kQueueCap));
  k_qinit<<<64, 256, 0, s>>>(qseq);
  launches += 1;
  ExtArgs A{};
  const hm_tuning tu = tuning();
  A.split_min = tu.split_min;
  A.pair_mode = tu.pair_mode;
  A.seeds_per_fetch = tu.seeds_per_fetch;
  A.poll_mask = (uint32_t)tu.poll_every - 1u;
  A.leaf_flatten = tu.leaf_flatten > 0 ? 1 : 0;
  A.wps_shift = wps_shift(tu);
  A.lookahead = tu.lookahead > 0 ? 1 : 0;
  A.seeds = seeds;
  A.nseeds = nseeds;
  A.qbuf = qbuf;
  A.qseq = qseq;
  A.ctl = ctl;
  A.rows = rows;
  A.cap = 0;
  A.root_mask = nullptr;
  A.budget_ns = budget_ms() * 1000000ull;
  A.max_chunks = budget_chunks();
  A.plans = d_plans;
  A.seed_pid = seed_pid;
  A.counts = d_counts;
  A.row_off = d_off;
  A.row_cap = d_cap;
  A.row_cursor = d_cursor;
  A.grp_slots = grp_slots;
  const int slot = min_blocks_slot(tu.extend_min_blocks);
  const size_t smem = warp_smem_bytes(grp_slots) * kExtWarps;
  const bool counters = counters_enabled();
  bool sym = false;
  for (const Plan &pl : plans) sym |= pl.naut > 1;
  const int grid = extend_grid<true>(want_rows, counters, smem, slot, false, sym);
  if (grid <= 0) return HM_ERR_CUDA;
  st.extend_grid = grid;
  st.extend_block = kExtThreads;
  NvtxRange r_ext("hm.batch_extend");
  Timer t_ext(s, timing);
  extend_kernel<true>(want_rows, counters, slot, false, sym)<<<grid, kExtThreads, smem, s>>>(G, plans[0], A);
  launches += 1;
  t_ext.stop();
  HM_CUDA_TRY(cudaGetLastError());
  Ctl h;
  std::vector<unsigned long long> hc(npat);
  HM_CUDA_TRY(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  HM_CUDA_TRY(cudaMemcpyAsync(hc.data(), d_counts, sizeof(unsigned long long) * npat,
                              cudaMemcpyDeviceToHost, s));
  HM_CUDA_TRY(cudaStreamSynchronize(s));
  st.ms_edge_scan = t_edge.ms();
  st.ms_overlap = t_ov.ms();
  st.ms_extend = t_ext.ms();
  st.seeds_scanned = (uint64_t)m;
  st.states_injected = any_ov ? h.nseeds : h.nseeds_raw;
  st.tasks_donated = h.donated;
  st.chunks = h.chunks;
  st.bytes_extend = h.bytes_extend;
  st.model_bytes_extend = h.bytes_extend_model;
  st.candidates = h.lanes;
  if (h.status == kStatBudget) return HM_ERR_BUDGET;
  if (h.status != kStatOk) return HM_ERR_CUDA;
  uint64_t total = 0;
  bool over = false;
  for (int32_t i = 0; i < npat; ++i) {
    counts[i] = hc[i];
    total += hc[i];
    if (want_rows && hc[i] > cap[i]) over = true;
  }
  st.matches = total;
  st.kernel_launches = launches;
  if (!want_rows) return HM_OK;
  if (over && !fit) return HM_ERR_CAPACITY;
  // ---- one sort for all patterns whose rows fit: key (pattern id, row), then back to each region
  std::vector<unsigned long long> start(npat + 1, 0);
  for (int32_t i = 0; i < npat; ++i) {
    const bool ok = hc[i] <= cap[i];
    if (fit) fit[i] = ok ? 1 : 0;
    start[i + 1] = start[i] + (ok ? hc[i] : 0);
  }
  total = start[npat];
  if (total == 0) return HM_OK;
  NvtxRange r_sort("hm.batch_sort_rows");
  Timer t_sort(s, timing);
  HM_CUDA_TRY(cudaMemcpyAsync(d_start, start.data(), sizeof(unsigned long long) * npat,
                              cudaMemcpyHostToDevice, s));
  const int width = kmax + 1;
  int32_t *packed, *tmp;
  HM_CUDA_TRY(sc.get((void **)&packed, sizeof(int32_t) * (size_t)total * width));
  HM_CUDA_TRY(sc.get((void **)&tmp, sizeof(int32_t) * (size_t)total * width));
  const int grid_r = (int)std::max<uint64_t>(1, std::min<uint64_t>((total + 255) / 256, (uint64_t)sms * 16));
  k_pack_rows<<<grid_r, 256, 0, s>>>(rows, d_off, d_start, d_ks, npat, total, width, packed);
  int cols[kMaxK + 1], bits[kMaxK + 1];
  uint32_t xr[kMaxK + 1];
  for (int c = 0; c < width; ++c) {
    cols[c] = c;
    bits[c] = c == 0 ? bits_for(npat) : bits_for(g->n);
    xr[c] = 0;
  }
  int nl = 0;
  hm_status r = radix_sort_rows_cols(packed, tmp, (int64_t)total, width, cols, bits, xr, width, s, &nl);
  if (r != HM_OK) return r;
  k_unpack_rows<<<grid_r, 256, 0, s>>>(packed, d_off, d_start, d_ks, total, width, rows);
  t_sort.stop();
  HM_CUDA_TRY(cudaGetLastError());
  st.kernel_launches += 2 + nl;
  if (timing) {
    HM_CUDA_TRY(cudaStreamSynchronize(s));
    st.ms_sort = t_sort.ms();
  }
  return HM_OK;
}

}  // namespace
}  // namespace hm

namespace hm {
hm_status enumerate_batch_fit(const hm_graph *g, const hm_pattern *const *patterns, const int32_t *modes,
                              int32_t npat, int32_t *rows_dev, const uint64_t *row_offsets, uint64_t *counts,
                              uint8_t *fit, cudaStream_t stream) {
  if (npat > 0 && (!rows_dev || !row_offsets || !fit)) return HM_ERR_ARG;
  return run_batch(g, patterns, modes, npat, rows_dev, row_offsets, counts, stream, fit);
}
}  // namespace hm

extern "C" hm_status hm_count_batch(const hm_graph *g, const hm_pattern *const *patterns,
                                    const int32_t *modes, int32_t npat, uint64_t *counts,
                                    void *stream) {
  return hm::run_batch(g, patterns, modes, npat, nullptr, nullptr, counts, (cudaStream_t)stream);
}

extern "C" hm_status hm_enumerate_batch(const hm_graph *g, const hm_pattern *const *patterns,
                                        const int32_t *modes, int32_t npat, int32_t *rows_dev,
                                        const uint64_t *row_offsets, uint64_t *counts,
                                        void *stream) {
  if (npat > 0 && (!rows_dev || !row_offsets)) return HM_ERR_ARG;
  return hm::run_batch(g, patterns, modes, npat, rows_dev, row_offsets, counts, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// hm_autotune: pick the extension kernel's launch knobs for a workload by
// timing candidate settings on its batched count (coordinate descent), with
// an optional cache file of earlier choices.
// ---------------------------------------------------------------------------
#include <chrono>
#include <cstdio>
#include <string>

namespace hm {
namespace {

// The knobs the tuner searches, each with its candidate values.
struct Dim {
  int32_t hm_tuning::*field;
  std::vector<int32_t> values;
};

std::vector<Dim> tune_dims() {
  return {
      {&hm_tuning::warps_per_state, {1, 2, 4}},
      {&hm_tuning::seeds_per_fetch, {1, 2, 4, 8, 16, 32, 64}},
      {&hm_tuning::arc_filter, {1, 16, -1}},  // intersection: filter probe / binary search in short lists / always
      {&hm_tuning::extend_min_blocks, {4, 5, 6}},
      {&hm_tuning::split_min, {16, 64, 256, 1024}},
      {&hm_tuning::poll_every, {32, 128, 512}},
      {&hm_tuning::pair_mode, {0, 1}},
      {&hm_tuning::leaf_flatten, {1, -1}},
      {&hm_tuning::lookahead, {-1, 1}},
  };
}

const char *kTuneFields[] = {"extend_min_blocks", "split_min", "pair_mode", "seeds_per_fetch", "poll_every",
                             "leaf_flatten", "arc_filter", "share_seeds", "symmetry", "warps_per_state",
                             "lookahead"};
int32_t hm_tuning::*const kTuneMembers[] = {
    &hm_tuning::extend_min_blocks, &hm_tuning::split_min, &hm_tuning::pair_mode, &hm_tuning::seeds_per_fetch,
    &hm_tuning::poll_every, &hm_tuning::leaf_flatten, &hm_tuning::arc_filter, &hm_tuning::share_seeds,
    &hm_tuning::symmetry, &hm_tuning::warps_per_state, &hm_tuning::lookahead};
constexpr int kNumTuneFields = 11;

// A fingerprint of the graph (sizes, directory sizes and a strided sample of
// its sorted arc arrays, FNV-1a) and of the workload (the multiset of pattern
// sizes and modes): the cache key of a tuned setting.
std::string tune_key(const hm_graph *g, const hm_pattern *const *patterns, const int32_t *modes, int32_t npat,
                     cudaStream_t s) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xff;
      h *= 1099511628211ull;
    }
  };
  mix((uint64_t)g->n);
  mix((uint64_t)g->m);
  mix((uint64_t)g->ndir_out);
  mix((uint64_t)g->ndir_in);
  constexpr int kSamples = 64, kRun = 16;
  std::vector<int32_t> buf(2 * kSamples * kRun, 0);
  if (g->m >= kRun) {
    for (int i = 0; i < kSamples; ++i) {
      const int64_t at = (g->m - kRun) * i / std::max(kSamples - 1, 1);
      cudaMemcpyAsync(buf.data() + 2 * i * kRun, g->src + at, sizeof(int32_t) * kRun, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(buf.data() + (2 * i + 1) * kRun, g->out_adj + at, sizeof(int32_t) * kRun,
                      cudaMemcpyDeviceToHost, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) (void)cudaGetLastError();
  }
  for (int32_t v : buf) mix((uint32_t)v);
  int hist[2][HM_MAX_K + 1] = {};
  for (int32_t i = 0; i < npat; ++i) hist[modes[i] ? 1 : 0][patterns[i]->k]++;
  std::string key;
  char tmp[64];
  std::snprintf(tmp, sizeof tmp, "g%016llx", (unsigned long long)h);
  key += tmp;
  for (int m = 0; m < 2; ++m)
    for (int k = 2; k <= HM_MAX_K; ++k)
      if (hist[m][k]) {
        std::snprintf(tmp, sizeof tmp, "_%c%dx%d", m ? 'i' : 'm', k, hist[m][k]);
        key += tmp;
      }
  return key;
}

// The last line of the cache file with this key: "<key> name=value ... ms=<t>".
bool cache_lookup(const char *path, const std::string &key, hm_tuning *t, float *ms) {
  FILE *f = std::fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    char k[256];
    int off = 0;
    if (std::sscanf(line, "%255s%n", k, &off) != 1 || key != k) continue;
    hm_tuning c{};
    float m = 0.f;
    int got = 0;
    const char *p = line + off;
    char name[64];
    double v;
    int n = 0;
    while (std::sscanf(p, " %63[a-z_]=%lf%n", name, &v, &n) == 2) {
      p += n;
      if (std::string(name) == "ms") {
        m = (float)v;
        continue;
      }
      for (int i = 0; i < kNumTuneFields; ++i)
        if (std::string(name) == kTuneFields[i]) {
          c.*kTuneMembers[i] = (int32_t)v;
          ++got;
        }
    }
    if (got == kNumTuneFields) {
      *t = c;
      *ms = m;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const char *path, const std::string &key, const hm_tuning &t, float ms) {
  FILE *f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s", key.c_str());
  for (int i = 0; i < kNumTuneFields; ++i) std::fprintf(f, " %s=%d", kTuneFields[i], t.*kTuneMembers[i]);
  std::fprintf(f, " ms=%.4f\n", ms);
  std::fclose(f);
}

}  // namespace
}  // namespace hm

extern "C" hm_status hm_autotune_cached(const hm_graph *g, const hm_pattern *const *patterns,
                                        const int32_t *modes, int32_t npat, uint32_t budget_ms,
                                        const char *cache_path, hm_tuning *best, float *best_ms,
                                        int32_t *from_cache, void *stream) {
  if (!g || !best || npat <= 0 || !patterns || !modes) return HM_ERR_ARG;
  for (int32_t i = 0; i < npat; ++i)
    if (!patterns[i]) return HM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (from_cache) *from_cache = 0;
  hm_tuning before{};
  hm_get_tuning(&before);
  std::string key;
  if (cache_path && *cache_path) {
    key = hm::tune_key(g, patterns, modes, npat, s);
    hm_tuning c{};
    float ms = 0.f;
    if (hm::cache_lookup(cache_path, key, &c, &ms) && hm_set_tuning(&c) == HM_OK) {
      hm_get_tuning(best);
      if (best_ms) *best_ms = ms;
      if (from_cache) *from_cache = 1;
      return HM_OK;
    }
  }
  std::vector<uint64_t> counts(npat), ref(npat);
  // reference run with the current knobs (also warms caches and the pool)
  hm_status st = hm::run_batch(g, patterns, modes, npat, nullptr, nullptr, ref.data(), s);
  if (st != HM_OK) return st;
  const auto t_start = std::chrono::steady_clock::now();
  auto spent_ms = [&] {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  };
  // best of two timed runs; a count that differs from the reference (which
  // no knob can cause) is reported as an error
  auto measure = [&](const hm_tuning &c, double *t_out) -> hm_status {
    hm_status r = hm_set_tuning(&c);
    if (r != HM_OK) return r;
    double t_min = 1e30;
    for (int rep = 0; rep < 2; ++rep) {
      const auto t0 = std::chrono::steady_clock::now();
      r = hm::run_batch(g, patterns, modes, npat, nullptr, nullptr, counts.data(), s);
      const auto t1 = std::chrono::steady_clock::now();
      if (r != HM_OK) return r;
      if (counts != ref) return HM_ERR_CUDA;
      t_min = std::min(t_min, std::chrono::duration<double, std::milli>(t1 - t0).count());
    }
    *t_out = t_min;
    return HM_OK;
  };
  hm_tuning pick{};
  hm_get_tuning(&pick);  // the current setting, defaults filled in
  double best_t = 0;
  st = measure(pick, &best_t);
  // coordinate descent: one knob at a time over its candidate values, keeping
  // a change only when it is faster by more than 1 %; passes repeat until one
  // changes nothing or the budget is spent
  const std::vector<hm::Dim> dims = hm::tune_dims();
  bool improved = true, out_of_time = false;
  for (int pass = 0; st == HM_OK && improved && !out_of_time && pass < 4; ++pass) {
    improved = false;
    for (const hm::Dim &d : dims) {
      if (st != HM_OK || out_of_time) break;
      for (int32_t v : d.values) {
        if (pick.*d.field == v) continue;
        hm_tuning c = pick;
        c.*d.field = v;
        double t = 0;
        st = measure(c, &t);
        if (st != HM_OK) break;
        if (t < best_t * 0.99) {
          best_t = t;
          pick = c;
          improved = true;
        }
        if (budget_ms && spent_ms() > (double)budget_ms) {
          out_of_time = true;
          break;
        }
      }
    }
  }
  if (st != HM_OK) {
    hm_set_tuning(&before);
    return st;
  }
  hm_set_tuning(&pick);
  hm_get_tuning(best);  // with the defaults filled in
  if (best_ms) *best_ms = (float)best_t;
  if (!key.empty()) hm::cache_store(cache_path, key, *best, (float)best_t);
  return HM_OK;
}

extern "C" hm_status hm_autotune(const hm_graph *g, const hm_pattern *const *patterns,
                                 const int32_t *modes, int32_t npat, uint32_t budget_ms,
                                 hm_tuning *best, float *best_ms, void *stream) {
  return hm_autotune_cached(g, patterns, modes, npat, budget_ms, nullptr, best, best_ms, nullptr, stream);
}
