// hm_kernels.cuh -- device code of the matching path, shared by the single-pattern
// (hm_match.cu) and batched (hm_batch.cu) entry points.  Each translation unit
// that includes it gets its own copy of these kernels.
//
//   k_edge_seed     every target arc is tried as the image of the reordered
//                   pattern arc between positions 0 and 1 (the loop "for all
//                   e in E2" of the HiPerMotif algorithm): vertex validator
//                   (Alg. 2) on the position-0 image, edge validator (Alg. 3)
//                   label, opposite-arc and degree checks.  Each block streams
//                   one contiguous span of the arcs in CSR order with int4
//                   loads (the next step's already in flight); survivors go
//                   through per-warp shared buffers into the seed queue.
//   k_seed_overlap  the edge validator's neighbour-overlap test
//                   |N_u & N_v| >= |N_0 & N_1|, one warp per surviving arc,
//                   launched only when the right side is non-zero.
//   k_extend        state injection and extension: each seed is a depth-2
//                   partial mapping; a persistent kernel extends it vertex by
//                   vertex, one warp per state.  At each depth the candidates
//                   are the shortest label-compatible anchor range (part of
//                   the out- or in-list of an already-mapped neighbour),
//                   scanned 32 at a time; each lane checks one candidate
//                   (injectivity, degrees, the other pattern arcs and the
//                   induced non-arcs through the arc filter and hash table,
//                   or a binary search for short lists) and a ballot gives
//                   the survivors.  The depth-first stack lives in shared
//                   memory.  At the last inner depth the survivors' leaf
//                   ranges are swept together (leaf_flatten).  Idle warps post
//                   donation requests; a busy warp claims one and splits off
//                   half of its shallowest unfinished range through a bounded
//                   lock-free queue.  Every wait is bounded by the call's time
//                   budget.  With a pendant position 1 the seeds of one
//                   position-0 image (induced: at most 32 of them) share one
//                   search, and position 1 is chosen at the leaves
//                   (expand_position1).  A pattern with label-preserving
//                   automorphisms is searched for one map per orbit (order
//                   constraints between images) and each map found is
//                   written with its automorphic images.
//   k_seed_rows     two-vertex patterns: each seed is already a match.
//
// Output: a match count (uint64), and optionally rows in original pattern
// order written at an atomic cursor and then radix-sorted lexicographically
// (hm_sort.cu), which makes the final order deterministic.
#pragma once

#include <cuda/atomic>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "hm_internal.cuh"

namespace hm {

void ensure_pool();

namespace {

constexpr int kExtThreads = 256;
constexpr int kExtWarps = kExtThreads / 32;
constexpr int kSeedThreads = 256;
constexpr uint32_t kFull = 0xffffffffu;
constexpr uint64_t kQueueCap = 1ull << 16;  // donated tasks in flight (power of two)

struct Task {
  int32_t depth;     // mapped positions (>= 2)
  int32_t drive;     // driving condition index for position `depth`
  uint32_t pmask;    // candidates allowed in the first chunk [lo, lo+32)
  int32_t pid;       // pattern of the task (batched launches)
  int32_t lo, hi;    // range of the driving list (absolute offsets)
  int32_t vlo, vhi;  // shared position-0 states: the group's seeds [vlo, vhi)
  int32_t map[kMaxK];
};
static_assert(sizeof(Task) == 32 + 4 * kMaxK && sizeof(Task) % 16 == 0, "task layout");
constexpr int kTaskWords = sizeof(Task) / 4;

// Control block of one call.  Words that different warps hit at high rates
// sit on separate 128-byte lines so they do not contend for one cache line.
struct Ctl {
  alignas(128) unsigned long long seed_next;  // next unclaimed seed
  alignas(128) unsigned long long head;       // donation queue
  unsigned long long tail;
  alignas(128) int32_t active;                // warps that hold work
  alignas(128) int32_t hungry;                // warps waiting for work
  int32_t requests;                           // donations asked for, not yet claimed
  alignas(128) int32_t status;
  alignas(128) unsigned long long nseeds_raw; // arcs passing the edge scan
  unsigned long long nseeds;                  // after the overlap test
  unsigned long long ngroups;                 // shared position-0 states
  unsigned long long count;
  unsigned long long rows_written;
  unsigned long long chunks;
  unsigned long long donated;
  // bytes of the instrumented launches: {requested, model} for each kernel
  unsigned long long bytes_edge, bytes_edge_model;
  unsigned long long bytes_overlap, bytes_overlap_model;
  unsigned long long bytes_extend, bytes_extend_model;
  unsigned long long lanes;                   // candidates examined (instrumented launches only)
  unsigned long long level_chunks[kMaxK];     // per depth (instrumented launches only)
  unsigned long long level_lanes[kMaxK];
};

struct ExtArgs {
  int32_t split_min;        // donate a range only while it holds at least this many candidates
  int32_t pair_mode;        // spread (candidate, condition) pairs over lanes on short ranges
  int32_t seeds_per_fetch;  // seeds a warp claims at once
  uint32_t poll_mask;       // a busy warp looks for donation requests every poll_mask+1 chunks
  int32_t leaf_flatten;     // run the last depth of all survivors of a chunk together
  int32_t wps_shift;        // log2 of the warps per depth-2 state: each state's first
                            // extension range is split into that many parts, one per claim
  const int2 *seeds;
  const unsigned long long *nseeds;
  Task *qbuf;
  unsigned long long *qseq;
  Ctl *ctl;
  int32_t *rows;
  unsigned long long cap;
  const uint8_t *root_mask;
  unsigned long long budget_ns;
  unsigned long long max_chunks;
  // batched launches (k_extend<..., kBatch = true>): one plan per pattern, the
  // pattern of each seed, and per-pattern counts and row regions
  const Plan *plans;
  const int32_t *seed_pid;
  unsigned long long *counts;
  const unsigned long long *row_off;  // first int32 of each pattern's rows in `rows`
  const unsigned long long *row_cap;  // rows each pattern may write
  unsigned long long *row_cursor;     // rows each pattern has claimed
  int32_t grp_slots;                  // group slots per warp (max over the patterns)
  int32_t lookahead;                  // apply the look-ahead classes at inner depths
  // shared position-0 states (single-pattern launches with P.defer1): one
  // int4 {u, first, end, 0} per distinct position-0 image instead of `seeds`,
  // and the seeds sorted by (u, v), whose .y over [first, end) are the
  // images position 1 may take
  const int4 *groups;
  const int2 *sorted_seeds;
};

using atomic_u64 = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>;
using atomic_i32 = cuda::atomic_ref<int32_t, cuda::thread_scope_device>;

__device__ __forceinline__ int32_t ld_volatile(const int32_t *p) {
  return *(const volatile int32_t *)p;
}

// Is a search over `len` sorted entries long enough to ask the arc filter first?
__device__ __forceinline__ bool use_filter(const DevGraph &G, int32_t len) {
  return G.filt_min >= 0 && len > G.filt_min;
}

// ---------------------------------------------------------------------------
// arc lookup: is (x -> y) an arc?  Searches the shorter of out(x) and in(y).
// ---------------------------------------------------------------------------
template <bool kC>
__device__ __forceinline__ bool arc_lookup(const DevGraph &G, int32_t x, int32_t y, int32_t outdeg_x,
                                           int32_t indeg_y, int32_t *lab, Bytes &ctr) {
  if (outdeg_x == 0 || indeg_y == 0) return false;
  if (use_filter(G, min(outdeg_x, indeg_y)))
    return arc_maybe<kC>(G, x, y, ctr) && arc_find<kC>(G, x, y, lab, ctr);
  if (kC) ctr += 8;
  if (outdeg_x <= indeg_y) {
    const int32_t o = __ldg(&G.off[HM_AT(G, x, G.n, kChkVertex)].x);
    const int32_t i = search_g<kC>(G, G.out_adj, o, outdeg_x, y, ctr);
    if (i < 0) return false;
    if (kC) ctr += 4;
    *lab = __ldg(G.out_elab + HM_AT(G, i, G.m, kChkList));
    return true;
  }
  const int32_t o = __ldg(&G.off[HM_AT(G, y, G.n, kChkVertex)].y);
  const int32_t i = search_g<kC>(G, G.in_adj, o, indeg_y, x, ctr);
  if (i < 0) return false;
  if (kC) ctr += 4;
  *lab = __ldg(G.in_elab + HM_AT(G, i, G.m, kChkList));
  return true;
}

// ---------------------------------------------------------------------------
// edge scan: vertex validator + edge validator (label, opposite arc, degrees)
// ---------------------------------------------------------------------------
// `fresh`: the previous arc of this thread had another source (consecutive
// arcs of one source share its record; the instrumented count takes it once).
template <bool kC>
__device__ __forceinline__ bool seed_test(const DevGraph &G, const Plan &P, int32_t a, int32_t b,
                                          int32_t l, const uint8_t *root_mask, int2 *out,
                                          Bytes &ctr, bool fresh = true) {
  if (l != P.seed_lab) return false;                       // match(e1, e2)
  const int32_t u = P.seed_rev ? b : a;                     // image of position 0
  const int32_t v = P.seed_rev ? a : b;                     // image of position 1
  if (kC && (fresh || P.seed_rev)) ctr += 16;
  if (kC) ctr.model += 12;
  const int4 iu = __ldg(&G.vi[HM_AT(G, u, G.n, kChkVertex)]);                          // Alg. 2 on u
  if (iu.x != P.vlab[0] || iu.y < P.dout[0] || iu.z < P.din[0]) return false;
  if (kC) {
    ctr += 16;
    ctr.model += 12;
  }
  const int4 iv = __ldg(&G.vi[HM_AT(G, v, G.n, kChkVertex)]);                          // match(v, 1) + degrees
  if (iv.x != P.vlab[1] || iv.y < P.dout[1] || iv.z < P.din[1]) return false;
  if (root_mask && ((P.root_pos == 0 && !root_mask[u]) || (P.root_pos == 1 && !root_mask[v])))
    return false;
  if (P.back_req | P.back_forbid) {
    // the arc opposite to the seeding one is (b -> a) in both seeding directions
    const int4 ib = P.seed_rev ? iu : iv;
    const int4 ia = P.seed_rev ? iv : iu;
    if (kC) ctr.model += search_bytes(min(ib.y, ia.z));
    if (P.back_req && use_filter(G, min(ib.y, ia.z)) && !arc_maybe_l<kC>(G, b, a, P.back_lab, ctr))
      return false;
    int32_t lab = 0;
    bool found = arc_lookup<kC>(G, b, a, ib.y, ia.z, &lab, ctr);
    if (P.back_req && (!found || lab != P.back_lab)) return false;
    if (P.back_forbid && found) return false;
  }
  *out = make_int2(u, v);
  if (kC) {
    ctr += 8;
    ctr.model += 8;
  }
  return true;
}

// Each block scans one contiguous span of the arcs, 1024 per step (128 per
// warp): each thread takes four consecutive arcs (one int4 of each stream) and
// already has the next step's three int4 loads in flight while it tests the
// current ones.  Survivors are appended to a per-warp buffer in shared memory
// (warp prefix sum) and flushed to the seed queue with one atomic per 32 or
// more seeds, so no block-wide barrier is needed, and seeds next to each other
// in the queue come from nearby arcs (mostly the same source), which keeps the
// extension kernel's concurrent warps on the same lists.  (One span per warp
// kept the seeds closer still but streamed 9,728 separate regions and was
// 1.7x slower on the 150M-arc graph.)
constexpr int kSeedBuf = 160;  // flushed at >= 32; one step adds at most 128

template <bool kC>
__global__ void __launch_bounds__(kSeedThreads)
k_edge_seed(const __grid_constant__ DevGraph G, const __grid_constant__ Plan P,
            const uint8_t *__restrict__ root_mask, int2 *__restrict__ seeds,
            unsigned long long cap, unsigned long long *__restrict__ nseeds,
            unsigned long long *__restrict__ bytes, int64_t e_begin, int64_t e_end) {
  Bytes ctr;
  __shared__ int2 s_buf[kSeedThreads / 32][kSeedBuf];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int2 *buf = s_buf[warp];
  int nbuf = 0;  // same in every lane of the warp
  // arcs [e_begin, e_end), e_begin a multiple of 4 so the int4 streams stay aligned
  const int64_t ngroups = (e_end - e_begin + 3) >> 2;
  const int64_t full_groups = (e_end - e_begin) >> 2;
  const int4 *src4 = reinterpret_cast<const int4 *>(G.src + e_begin);
  const int4 *dst4 = reinterpret_cast<const int4 *>(G.out_adj + e_begin);
  const int4 *lab4 = reinterpret_cast<const int4 *>(G.out_elab + e_begin);
  const int64_t span = ((ngroups + gridDim.x - 1) / gridDim.x + kSeedThreads - 1) / kSeedThreads *
                       kSeedThreads;  // groups per block
  const int64_t g_begin = (int64_t)blockIdx.x * span, g_end = min(ngroups, g_begin + span);
  int4 na = make_int4(0, 0, 0, 0), nb = na, nl = na;
  {
    const int64_t g0 = g_begin + threadIdx.x;
    if (g0 < g_end && g0 < full_groups) {
      na = __ldcs(src4 + g0);
      nb = __ldcs(dst4 + g0);
      nl = __ldcs(lab4 + g0);
    }
  }
  for (int64_t base = g_begin; base < g_end; base += kSeedThreads) {
    const int64_t gi = base + threadIdx.x;
    const int4 a = na, b = nb, l = nl;
    if (gi + kSeedThreads < g_end && gi + kSeedThreads < full_groups) {  // next step's arcs
      na = __ldcs(src4 + gi + kSeedThreads);
      nb = __ldcs(dst4 + gi + kSeedThreads);
      nl = __ldcs(lab4 + gi + kSeedThreads);
    }
    int2 s[4];
    bool ok[4] = {false, false, false, false};
    if (gi >= g_end) {
      // past this warp's span
    } else if (gi < full_groups) {
      if (kC) {
        ctr += 48;
        ctr.model += 48;
      }
      ok[0] = seed_test<kC>(G, P, a.x, b.x, l.x, root_mask, &s[0], ctr);
      ok[1] = seed_test<kC>(G, P, a.y, b.y, l.y, root_mask, &s[1], ctr, a.y != a.x);
      ok[2] = seed_test<kC>(G, P, a.z, b.z, l.z, root_mask, &s[2], ctr, a.z != a.y);
      ok[3] = seed_test<kC>(G, P, a.w, b.w, l.w, root_mask, &s[3], ctr, a.w != a.z);
    } else if (gi < ngroups) {
      for (int j = 0; j < 4; ++j) {
        const int64_t e = e_begin + gi * 4 + j;
        if (kC && e < e_end) {
          ctr += 12;
          ctr.model += 12;
        }
        if (e < e_end)
          ok[j] = seed_test<kC>(G, P, G.src[HM_AT(G, e, G.m, kChkList)], G.out_adj[HM_AT(G, e, G.m, kChkList)],
                                G.out_elab[HM_AT(G, e, G.m, kChkList)], root_mask, &s[j], ctr);
      }
    }
    const uint32_t cnt = (uint32_t)ok[0] + ok[1] + ok[2] + ok[3];
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    int at = nbuf + (int)(incl - cnt);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (ok[j]) buf[at++] = s[j];
    nbuf += (int)__shfl_sync(kFull, incl, 31);
    __syncwarp();
    if (nbuf >= 32) {
      unsigned long long off = 0;
      if (lane == 0) off = atomicAdd(nseeds, (unsigned long long)nbuf);
      off = __shfl_sync(kFull, off, 0);
      for (int i = lane; i < nbuf; i += 32)
        if (off + i < cap) seeds[off + i] = buf[i];
      nbuf = 0;
      __syncwarp();
    }
  }
  if (nbuf) {
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(nseeds, (unsigned long long)nbuf);
    off = __shfl_sync(kFull, off, 0);
    for (int i = lane; i < nbuf; i += 32)
      if (off + i < cap) seeds[off + i] = buf[i];
  }
  if (kC) {
    for (int o = 16; o; o >>= 1) {
      ctr.req += __shfl_xor_sync(kFull, ctr.req, o);
      ctr.model += __shfl_xor_sync(kFull, ctr.model, o);
    }
    if (lane == 0 && ctr.req) atomicAdd(bytes, (unsigned long long)ctr.req);
    if (lane == 0 && ctr.model) atomicAdd(bytes + 1, (unsigned long long)ctr.model);
  }
}

// ---------------------------------------------------------------------------
// neighbour-overlap test, one warp per seed
// ---------------------------------------------------------------------------

// Is w a neighbour (in or out) of y?
template <bool kC>
__device__ __forceinline__ bool in_nbhd(const DevGraph &G, int32_t y, int4 iy, int2 oy,
                                        int32_t w, Bytes &ctr) {
  int32_t lab;
  if (iy.y && (use_filter(G, iy.y) ? arc_maybe<kC>(G, y, w, ctr) && arc_find<kC>(G, y, w, &lab, ctr)
                                   : search_g<kC>(G, G.out_adj, oy.x, iy.y, w, ctr) >= 0))
    return true;
  return iy.z && (use_filter(G, iy.z) ? arc_maybe<kC>(G, w, y, ctr) && arc_find<kC>(G, w, y, &lab, ctr)
                                      : search_g<kC>(G, G.in_adj, oy.y, iy.z, w, ctr) >= 0);
}

// In batched launches (kB) each seed carries its pattern id; the threshold is
// that pattern's, and seeds of patterns without an overlap test pass through.
template <bool kC, bool kB = false>
__global__ void __launch_bounds__(kSeedThreads)
k_seed_overlap(const __grid_constant__ DevGraph G, int32_t need_all, const int2 *__restrict__ in,
               const unsigned long long *__restrict__ nin, int2 *__restrict__ out,
               unsigned long long cap, unsigned long long *__restrict__ nout,
               unsigned long long *__restrict__ bytes, const Plan *__restrict__ plans = nullptr,
               const int32_t *__restrict__ pid_in = nullptr, int32_t *__restrict__ pid_out = nullptr) {
  Bytes ctr;
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_in = (int64_t)*nin;
  for (int64_t s = wid; s < n_in; s += nw) {
    const int2 uv = in[s];
    const int32_t pid = kB ? pid_in[s] : 0;
    const int32_t need = kB ? plans[pid].ov_need : need_all;
    if (kC && lane == 0) ctr += 72;
    int4 iu = __ldg(&G.vi[HM_AT(G, uv.x, G.n, kChkVertex)]), iv = __ldg(&G.vi[HM_AT(G, uv.y, G.n, kChkVertex)]);
    if (kC && lane == 0) ctr.model += 24 + 4ull * (iu.y + iu.z + iv.y + iv.z);  // a merge of the four lists
    int2 ou = __ldg(&G.off[HM_AT(G, uv.x, G.n, kChkVertex)]), ov = __ldg(&G.off[HM_AT(G, uv.y, G.n, kChkVertex)]);
    // iterate the side with fewer incident arcs, probe the other
    const bool swap = (iu.y + iu.z) > (iv.y + iv.z);
    const int4 ix = swap ? iv : iu, iy = swap ? iu : iv;
    const int2 ox = swap ? ov : ou, oy = swap ? ou : ov;
    const int32_t y = swap ? uv.x : uv.y;
    int32_t got = 0;
    // out-neighbours of x
    for (int32_t b = 0; b < ix.y && got < need; b += 32) {
      bool hit = false;
      if (b + lane < ix.y) {
        int32_t w = __ldg(G.out_adj + HM_AT(G, (int64_t)ox.x + b + lane, G.m, kChkList));
        if (kC) ctr += 4;
        hit = in_nbhd<kC>(G, y, iy, oy, w, ctr);
      }
      got += __popc(__ballot_sync(kFull, hit));
    }
    // in-neighbours of x that are not also out-neighbours
    for (int32_t b = 0; b < ix.z && got < need; b += 32) {
      bool hit = false;
      if (b + lane < ix.z) {
        int32_t w = __ldg(G.in_adj + HM_AT(G, (int64_t)ox.y + b + lane, G.m, kChkList));
        if (kC) ctr += 4;
        bool dup = ix.y && search_g<kC>(G, G.out_adj, ox.x, ix.y, w, ctr) >= 0;
        hit = !dup && in_nbhd<kC>(G, y, iy, oy, w, ctr);
      }
      got += __popc(__ballot_sync(kFull, hit));
    }
    if (got >= need && lane == 0) {
      unsigned long long at = atomicAdd(nout, 1ull);
      if (at < cap) {
        out[at] = uv;
        if (kB) pid_out[at] = pid;
      }
      if (kC) {
        ctr += 8;
        ctr.model += 8;
      }
    }
  }
  if (kC) {
    for (int o = 16; o; o >>= 1) {
      ctr.req += __shfl_xor_sync(kFull, ctr.req, o);
      ctr.model += __shfl_xor_sync(kFull, ctr.model, o);
    }
    if (lane == 0 && ctr.req) atomicAdd(bytes, (unsigned long long)ctr.req);
    if (lane == 0 && ctr.model) atomicAdd(bytes + 1, (unsigned long long)ctr.model);
  }
}

// ---------------------------------------------------------------------------
// persistent extension kernel
// ---------------------------------------------------------------------------

// The survivor (image of depth L) a flattened leaf candidate belongs to.
struct LeafOwner {
  int32_t c, off_out, off_in, deg_out, deg_in;
  int2 own[2];  // label group of the leaf inside c's out-list [0] / in-list [1]
};

struct WarpState {
  int32_t map[kMaxK];       // image of each mapped position
  int32_t deg_out[kMaxK];   // its out-degree
  int32_t deg_in[kMaxK];    // its in-degree
  int32_t off_out[kMaxK];   // its first out-arc
  int32_t off_in[kMaxK];    // its first in-arc
  int4 dir[kMaxK];          // its directory spans {out first, out count, in first, in count}
  int32_t lo[kMaxK];        // next chunk of the driving group at each depth
  int32_t hi[kMaxK];        // end of the driving range
  int32_t base[kMaxK];      // start of the chunk whose survivors are pending
  uint32_t mask[kMaxK];     // pending survivors of that chunk
  int32_t drive[kMaxK];     // driving condition at each depth
  int32_t vlo, vhi;         // shared position-0 states: the group's seeds
  // control state touched once per task or per 64 chunks (kept here, not in
  // registers): the call's deadline, the seed count, this warp's claimed
  // seeds [seed_at, seed_end), its match count and, for lane 0, the chunk
  // count already reported and the last polled status and request words
  unsigned long long deadline, nseeds, seed_at, seed_end, my_count;
  uint32_t chunks_flushed;  // chunk counts run modulo 2^32 and are compared by difference
  int32_t requests_seen, status_seen;
  // the current task's output: row cursor, first row, rows it may write
  unsigned long long *row_cursor;
  int32_t *row_base;
  unsigned long long row_cap;
  // the survivors whose leaf ranges a flattened sweep covers (leaf_flatten),
  // read by the lanes whose candidates they own
  LeafOwner owners[32];
  int4 owner_drive[32];     // {driving condition, range start, its kind, offset in the sweep}
  int4 owner_probe[32];     // {anchor, flags, arc label, group length}: the owner's first
                            // other positive condition, tested by the filter before the rest
                            // (flags: 1 valid, 2 arc anchor -> candidate, condition index << 8)
  Task stage;               // task being donated or received
};
// Each warp's WarpState is followed in shared memory by one int2 per positive
// condition of the pattern, {first, length} of the matching label group inside
// the anchor's list (first relative to the list start); Plan::gbase[p] indexes it.

template <bool kC>
__device__ __forceinline__ void set_mapped(const DevGraph &G, WarpState &S, int pos, int32_t c,
                                           int lane, Bytes &ctr) {
  if (kC && lane == 0) ctr += 48;
  // three independent 16-byte loads, each lane writing its own record's fields
  const bool known = c >= 0;  // c < 0: position 1 of a shared position-0 state, not yet chosen
  if (lane == 0) {
    const int4 vi = known ? __ldg(&G.vi[HM_AT(G, c, G.n, kChkVertex)]) : make_int4(0, 0, 0, 0);
    S.map[pos] = c;
    S.deg_out[pos] = vi.y;
    S.deg_in[pos] = vi.z;
  } else if (lane == 1) {
    const int2 o = known ? __ldg(&G.off[HM_AT(G, c, G.n, kChkVertex)]) : make_int2(0, 0);
    S.off_out[pos] = o.x;
    S.off_in[pos] = o.y;
  } else if (lane == 2) {
    S.dir[pos] = known ? __ldg(&G.vdir[HM_AT(G, c, G.n, kChkVertex)]) : make_int4(0, 0, 0, 0);
  }
}

// Symmetry breaking (Plan::naut > 1): candidate c for position p keeps the
// order constraints against earlier positions; position L's image is lc when
// it is not yet in S.map (the flattened leaf), otherwise pass L = p.
__device__ __noinline__ bool sym_ok(const Plan &P, const WarpState &S, int p, int32_t c, int L = -1,
                                    int32_t lc = 0) {
  uint32_t g = P.sym_gt[p], l = P.sym_lt[p];
  while (g) {
    const int q = __ffs(g) - 1;
    g &= g - 1;
    if (c <= (q == L ? lc : S.map[q])) return false;
  }
  while (l) {
    const int q = __ffs(l) - 1;
    l &= l - 1;
    if (c >= (q == L ? lc : S.map[q])) return false;
  }
  return true;
}

// The rows of one found map and of its automorphic images, P.naut rows from
// row r on: image s of original vertex v is the vertex at position
// P.aut[s][v].  Positions below `nmapped` are in map[]; position nmapped is
// e1 and the one after it e2.  Out of line: only symmetric patterns use it.
__device__ __noinline__ void write_match_rows(const Plan &P, int32_t *row_base, unsigned long long r,
                                              unsigned long long row_cap, const int32_t *map, int nmapped,
                                              int32_t e1, int32_t e2) {
  const int k = P.k;
  for (int s = 0; s < P.naut && r + s < row_cap; ++s) {
    int32_t *row = row_base + (r + s) * k;
    for (int v = 0; v < k; ++v) {
      const int i = P.aut[s][v];
      row[v] = i < nmapped ? map[i] : (i == nmapped ? e1 : e2);
    }
  }
}

// Look-ahead: candidate c for position p has, in every class of P.la[p]
// (direction, arc label, neighbour label), at least as many neighbours as
// the later positions of that class need -- their images must be distinct
// neighbours of c.  Out of line: only the look-ahead knob uses it.
template <bool kC>
__device__ __noinline__ bool lookahead_ok(const DevGraph &G, const Plan &P, int p, int32_t c, Bytes &ctr) {
  if (kC) ctr += 16;
  const int4 vd = __ldg(&G.vdir[HM_AT(G, c, G.n, kChkVertex)]);
  for (int j = 0; j < P.nla[p]; ++j) {
    const LookClass lc = P.la[p][j];
    const int4 *dir = lc.kind == kOut ? G.gdir_out : G.gdir_in;
    const int32_t first = lc.kind == kOut ? vd.x : vd.z, cnt = lc.kind == kOut ? vd.y : vd.w;
    int32_t len = 0;
    for (int32_t e = 0; e < cnt; ++e) {
      if (kC) ctr += 16;
      const int4 ent = __ldg(dir + HM_AT(G, (int64_t)first + e, lc.kind == kOut ? G.ndir_out : G.ndir_in,
                                         lc.kind == kOut ? kChkDirOut : kChkDirIn));
      if (ent.x == lc.alab && ent.y == lc.vlab) {
        len = ent.w - ent.z;
        break;
      }
    }
    if (len < lc.need) return false;
  }
  return true;
}

// Find the group (arc label, vertex label) in a directory span; {first, length} or {0, 0}.
template <bool kC>
__device__ __forceinline__ int2 dir_lookup(const DevGraph &G, const int4 *__restrict__ dir, int32_t first,
                                           int32_t cnt, int32_t alab, int32_t vlab, int lane, Bytes &ctr) {
  for (int32_t b = 0; b < cnt; b += 32) {
    int4 e = make_int4(0, 0, 0, 0);
    bool hit = false;
    if (b + lane < cnt) {
      if (kC) ctr += 16;
      e = __ldg(dir + HM_AT(G, (int64_t)first + b + lane, dir == G.gdir_out ? G.ndir_out : G.ndir_in,
                            dir == G.gdir_out ? kChkDirOut : kChkDirIn));
      hit = e.x == alab && e.y == vlab;
    }
    const uint32_t m = __ballot_sync(kFull, hit);
    if (m) {
      const int src = __ffs(m) - 1;
      const int32_t s0 = __shfl_sync(kFull, e.z, src), s1 = __shfl_sync(kFull, e.w, src);
      return make_int2(s0, s1 - s0);
    }
  }
  return make_int2(0, 0);
}

// Look up the label group of every anchor of position p; unless `keep`, pick the
// smallest group as the driving range.
template <bool kC>
__device__ __forceinline__ void setup_level(const DevGraph &G, const Plan &P, WarpState &S,
                                            int2 *__restrict__ grp, int p, int lane, bool keep,
                                            Bytes &ctr) {
  int best = 0;
  int32_t best_len = INT32_MAX;
  for (int j = 0; j < P.npos[p]; ++j) {
    const Cons cs = P.cons[p][j];
    const int4 d = S.dir[cs.q];
    const int2 r = cs.kind == kOut ? dir_lookup<kC>(G, G.gdir_out, d.x, d.y, cs.lab, P.vlab[p], lane, ctr)
                                   : dir_lookup<kC>(G, G.gdir_in, d.z, d.w, cs.lab, P.vlab[p], lane, ctr);
    if (lane == 0) grp[P.gbase[p] + j] = r;
    if (r.y < best_len) {
      best_len = r.y;
      best = j;
    }
  }
  if (lane == 0 && !keep) {
    const Cons cs = P.cons[p][best];
    const int2 r = grp[P.gbase[p] + best];
    const int32_t lo = (cs.kind == kOut ? S.off_out[cs.q] : S.off_in[cs.q]) + r.x;
    S.drive[p] = best;
    S.lo[p] = lo;
    S.hi[p] = lo + r.y;
    S.mask[p] = 0;
  }
}

// Does candidate c (taken from the driving group, so its arc label and vertex
// label already match) satisfy every other condition of position p?
template <bool kC, bool kSym>
__device__ __forceinline__ bool check_candidate(const DevGraph &G, const Plan &P,
                                                const WarpState &S, const int2 *__restrict__ grp,
                                                int p, int drive, int32_t c, bool leaf,
                                                const uint8_t *root_mask, Bytes &ctr) {
  for (int i = 0; i < p; ++i)
    if (S.map[i] == c) return false;                        // injective
  if (root_mask && p == P.root_pos && !root_mask[c]) return false;
  if (kSym && (P.sym_gt[p] | P.sym_lt[p]) && !sym_ok(P, S, p, c)) return false;
  const int nc = P.ncons[p];
  // c's own degrees: needed for the degree filter (inner levels) and to search
  // c's shorter list instead of a hub's; its offsets only for such a search
  const bool need_c = !leaf || nc > 1;
  int4 vi = make_int4(0, 0, 0, 0);
  int2 oc = make_int2(-1, -1);
  if (need_c) {
    if (kC) ctr += 16;
    vi = __ldg(&G.vi[HM_AT(G, c, G.n, kChkVertex)]);
    if (!leaf && (vi.y < P.dout[p] || vi.z < P.din[p])) return false;
  }
  for (int j = 0; j < nc; ++j) {
    if (j == drive) continue;
    const Cons cs = P.cons[p][j];
    const int q = cs.q;
    const int32_t fq = S.map[q];
    const bool fwd = cs.kind == kOut || cs.kind == kNotOut;   // arc f(q) -> c ?
    const int32_t x = fwd ? fq : c, y = fwd ? c : fq;         // the arc in question, x -> y
    bool found;
    int32_t lab;
    if (cs.kind <= kIn) {
      // positive: c in the (label, label) group of f(q), or f(q) in c's reverse list
      const int2 r = grp[P.gbase[p] + j];
      const int32_t rev_len = fwd ? vi.z : vi.y;
      if (r.y == 0 || rev_len == 0) return false;
      if (kC) ctr.model += search_bytes(min(rev_len, r.y));
      if (use_filter(G, min(rev_len, r.y))) {
        found = arc_maybe_l<kC>(G, x, y, cs.lab, ctr) && arc_find<kC>(G, x, y, &lab, ctr) && lab == cs.lab;
      } else if (rev_len < r.y) {
        if (oc.x < 0) {
          if (kC) ctr += 8;
          oc = __ldg(&G.off[HM_AT(G, c, G.n, kChkVertex)]);
        }
        const int32_t i = fwd ? search_g<kC>(G, G.in_adj, oc.y, rev_len, fq, ctr)
                              : search_g<kC>(G, G.out_adj, oc.x, rev_len, fq, ctr);
        if (kC && i >= 0) ctr += 4;
        found = i >= 0 && __ldg((fwd ? G.in_elab : G.out_elab) + HM_AT(G, i, G.m, kChkList)) == cs.lab;
      } else {
        const int32_t base = (fwd ? S.off_out[q] : S.off_in[q]) + r.x;
        found = search_g<kC>(G, fwd ? G.gout_adj : G.gin_adj, base, r.y, c, ctr) >= 0;
      }
      if (!found) return false;
    } else {
      // induced: no arc at all between f(q) and c in this direction
      const int32_t la = fwd ? S.deg_out[q] : S.deg_in[q];
      const int32_t lb = fwd ? vi.z : vi.y;
      if (la == 0 || lb == 0) continue;
      if (kC) ctr.model += search_bytes(min(la, lb));
      if (use_filter(G, min(la, lb))) {
        found = arc_maybe<kC>(G, x, y, ctr) && arc_find<kC>(G, x, y, &lab, ctr);
      } else if (la <= lb) {
        found = search_g<kC>(G, fwd ? G.out_adj : G.in_adj, fwd ? S.off_out[q] : S.off_in[q], la, c, ctr) >= 0;
      } else {
        if (oc.x < 0) {
          if (kC) ctr += 8;
          oc = __ldg(&G.off[HM_AT(G, c, G.n, kChkVertex)]);
        }
        found = search_g<kC>(G, fwd ? G.in_adj : G.out_adj, fwd ? oc.y : oc.x, lb, fq, ctr) >= 0;
      }
      if (found) return false;
    }
  }
  return true;
}

// One condition j of position p on candidate c (the j-th entry of cons[p]).
// The lane with `base` set also applies the per-candidate checks
// (injectivity, root mask, degree filter on inner levels).
template <bool kC, bool kSym>
__device__ __noinline__ bool check_one(const DevGraph &G, const Plan &P, const WarpState &S,
                                          const int2 *__restrict__ grp, int p, int j, int32_t c,
                                          bool base, bool leaf, const uint8_t *root_mask,
                                          Bytes &ctr) {
  if (base) {
    for (int i = 0; i < p; ++i)
      if (S.map[i] == c) return false;
    if (root_mask && p == P.root_pos && !root_mask[c]) return false;
    if (kSym && (P.sym_gt[p] | P.sym_lt[p]) && !sym_ok(P, S, p, c)) return false;
  }
  if (kC) ctr += 16;
  const int4 vi = __ldg(&G.vi[HM_AT(G, c, G.n, kChkVertex)]);
  if (base && !leaf && (vi.y < P.dout[p] || vi.z < P.din[p])) return false;
  const Cons cs = P.cons[p][j];
  const int q = cs.q;
  const int32_t fq = S.map[q];
  const bool fwd = cs.kind == kOut || cs.kind == kNotOut;
  const int32_t x = fwd ? fq : c, y = fwd ? c : fq;  // the arc in question, x -> y
  int32_t lab;
  if (cs.kind <= kIn) {
    const int2 r = grp[P.gbase[p] + j];
    const int32_t rev_len = fwd ? vi.z : vi.y;
    if (r.y == 0 || rev_len == 0) return false;
    if (kC) ctr.model += search_bytes(min(rev_len, r.y));
    if (use_filter(G, min(rev_len, r.y)))
      return arc_maybe_l<kC>(G, x, y, cs.lab, ctr) && arc_find<kC>(G, x, y, &lab, ctr) && lab == cs.lab;
    if (rev_len < r.y) {
      if (kC) ctr += 16;
      const int2 oc = __ldg(&G.off[HM_AT(G, c, G.n, kChkVertex)]);
      const int32_t i = fwd ? search_g<kC>(G, G.in_adj, oc.y, rev_len, fq, ctr)
                            : search_g<kC>(G, G.out_adj, oc.x, rev_len, fq, ctr);
      if (kC && i >= 0) ctr += 4;
      return i >= 0 && __ldg((fwd ? G.in_elab : G.out_elab) + HM_AT(G, i, G.m, kChkList)) == cs.lab;
    }
    const int32_t lo = (fwd ? S.off_out[q] : S.off_in[q]) + r.x;
    return search_g<kC>(G, fwd ? G.gout_adj : G.gin_adj, lo, r.y, c, ctr) >= 0;
  }
  const int32_t la = fwd ? S.deg_out[q] : S.deg_in[q];
  const int32_t lb = fwd ? vi.z : vi.y;
  if (la == 0 || lb == 0) return true;
  if (kC) ctr.model += search_bytes(min(la, lb));
  if (use_filter(G, min(la, lb))) return !(arc_maybe<kC>(G, x, y, ctr) && arc_find<kC>(G, x, y, &lab, ctr));
  if (la <= lb)
    return search_g<kC>(G, fwd ? G.out_adj : G.in_adj, fwd ? S.off_out[q] : S.off_in[q], la, c, ctr) < 0;
  if (kC) ctr += 16;
  const int2 oc = __ldg(&G.off[HM_AT(G, c, G.n, kChkVertex)]);
  return search_g<kC>(G, fwd ? G.in_adj : G.out_adj, fwd ? oc.y : oc.x, lb, fq, ctr) < 0;
}

// ---- last-level flattening ---------------------------------------------------
//
// At the last inner depth L = k-2, the survivors of a chunk (up to 32, one per
// lane) are not descended into one by one.  Each survivor lane looks up its
// own label groups and picks its own shortest anchor range for the leaf; the
// ranges are concatenated (warp prefix sum) and swept in full 32-lane chunks,
// each lane finding its survivor by a binary search over the prefix sums.
// Survivors whose leaf range exceeds kFlatMax stay pending for the ordinary
// descent, where their range can be split and donated.
constexpr int32_t kFlatMax = 2048;


// check_leaf's conditions without the arc filter (arc_filter = -1): each one
// searches the shorter of f(q)'s list and d's reverse list.  Out of line: the
// default path never runs it.
template <bool kC>
__device__ __noinline__ bool check_leaf_searched(const DevGraph &G, const Plan &P, const WarpState &S,
                                                 const int2 *__restrict__ grp, int p, int drive, int32_t d,
                                                 const LeafOwner &o, Bytes &ctr) {
  const int L = p - 1;
  const int nc = P.ncons[p];
  if (kC) ctr += 32;
  const int4 vi = __ldg(&G.vi[HM_AT(G, d, G.n, kChkVertex)]);
  const int2 od = __ldg(&G.off[HM_AT(G, d, G.n, kChkVertex)]);
  for (int j = 0; j < nc; ++j) {
    if (j == drive) continue;
    const Cons cs = P.cons[p][j];
    const int q = cs.q;
    const bool mine = q == L;
    const int32_t fq = mine ? o.c : S.map[q];
    const int32_t q_off_out = mine ? o.off_out : S.off_out[q];
    const int32_t q_off_in = mine ? o.off_in : S.off_in[q];
    const bool fwd = cs.kind == kOut || cs.kind == kNotOut;   // arc f(q) -> d ?
    if (cs.kind <= kIn) {
      const int2 r = mine ? (cs.kind == kOut ? o.own[0] : o.own[1]) : grp[P.gbase[p] + j];
      const int32_t rev_len = fwd ? vi.z : vi.y;
      if (r.y == 0 || rev_len == 0) return false;
      if (kC) ctr.model += search_bytes(min(rev_len, r.y));
      bool found;
      if (rev_len < r.y) {
        const int32_t i = fwd ? search_g<kC>(G, G.in_adj, od.y, rev_len, fq, ctr)
                              : search_g<kC>(G, G.out_adj, od.x, rev_len, fq, ctr);
        if (kC && i >= 0) ctr += 4;
        found = i >= 0 && __ldg((fwd ? G.in_elab : G.out_elab) + HM_AT(G, i, G.m, kChkList)) == cs.lab;
      } else {
        found = search_g<kC>(G, fwd ? G.gout_adj : G.gin_adj, (fwd ? q_off_out : q_off_in) + r.x, r.y,
                             d, ctr) >= 0;
      }
      if (!found) return false;
    } else {
      const int32_t la = fwd ? (mine ? o.deg_out : S.deg_out[q]) : (mine ? o.deg_in : S.deg_in[q]);
      const int32_t lb = fwd ? vi.z : vi.y;
      if (la == 0 || lb == 0) continue;
      if (kC) ctr.model += search_bytes(min(la, lb));
      const bool found =
          la <= lb ? search_g<kC>(G, fwd ? G.out_adj : G.in_adj, fwd ? q_off_out : q_off_in, la, d, ctr) >= 0
                   : search_g<kC>(G, fwd ? G.in_adj : G.out_adj, fwd ? od.y : od.x, lb, fq, ctr) >= 0;
      if (found) return false;
    }
  }
  return true;
}

// `first`: a positive condition whose filter probe the caller has already
// passed (-1: none); its exact lookup still follows.
template <bool kC, bool kSym>
__device__ __forceinline__ bool check_leaf(const DevGraph &G, const Plan &P, const WarpState &S,
                                           const int2 *__restrict__ grp, int p, int drive, int first,
                                           int32_t d, const LeafOwner &o, const uint8_t *root_mask,
                                           Bytes &ctr) {
  const int L = p - 1;
  if (d == o.c) return false;
  for (int i = 0; i < L; ++i)
    if (S.map[i] == d) return false;                        // injective
  if (root_mask && p == P.root_pos && !root_mask[d]) return false;
  if (kSym && (P.sym_gt[p] | P.sym_lt[p]) && !sym_ok(P, S, p, d, L, o.c)) return false;
  const int nc = P.ncons[p];
  if (nc <= 1) return true;
  if (G.filt_min >= 0) {
    // first the arc filter, which needs only the two endpoints: most candidates
    // fail a positive condition here, and most induced non-arcs are settled
    uint64_t settled = 0;
    for (int j = 0; j < nc; ++j) {
      if (j == drive || j == first) continue;
      const Cons cs = P.cons[p][j];
      const bool mine = cs.q == L;
      const int32_t fq = mine ? o.c : S.map[cs.q];
      const bool fwd = cs.kind == kOut || cs.kind == kNotOut;
      if (cs.kind <= kIn) {
        const int2 r = mine ? (cs.kind == kOut ? o.own[0] : o.own[1]) : grp[P.gbase[p] + j];
        if (r.y == 0) return false;
        if (kC) ctr.model += search_bytes(r.y);
        if (use_filter(G, r.y) && !arc_maybe_l<kC>(G, fwd ? fq : d, fwd ? d : fq, cs.lab, ctr))
          return false;
      } else {
        const int32_t la = fwd ? (mine ? o.deg_out : S.deg_out[cs.q]) : (mine ? o.deg_in : S.deg_in[cs.q]);
        if (kC) ctr.model += search_bytes(la);
        if (la == 0 || (use_filter(G, la) && !arc_maybe<kC>(G, fwd ? fq : d, fwd ? d : fq, ctr)))
          settled |= 1ull << j;
      }
    }
    // then the exact answers: short lists of f(q) are searched, the rest
    // looked up in the arc hash table -- d's own record is never needed
    for (int j = 0; j < nc; ++j) {
      if (j == drive || ((settled >> j) & 1)) continue;
      const Cons cs = P.cons[p][j];
      const int q = cs.q;
      const bool mine = q == L;
      const int32_t fq = mine ? o.c : S.map[q];
      const bool fwd = cs.kind == kOut || cs.kind == kNotOut;
      const int32_t x = fwd ? fq : d, y = fwd ? d : fq;
      int32_t lab;
      if (cs.kind <= kIn) {
        const int2 r = mine ? (cs.kind == kOut ? o.own[0] : o.own[1]) : grp[P.gbase[p] + j];
        const bool found =
            use_filter(G, r.y)
                ? arc_find<kC>(G, x, y, &lab, ctr) && lab == cs.lab
                : search_g<kC>(G, fwd ? G.gout_adj : G.gin_adj,
                               (fwd ? (mine ? o.off_out : S.off_out[q]) : (mine ? o.off_in : S.off_in[q])) + r.x,
                               r.y, d, ctr) >= 0;
        if (!found) return false;
      } else {
        const int32_t la = fwd ? (mine ? o.deg_out : S.deg_out[q]) : (mine ? o.deg_in : S.deg_in[q]);
        const bool found =
            use_filter(G, la)
                ? arc_find<kC>(G, x, y, &lab, ctr)
                : search_g<kC>(G, fwd ? G.out_adj : G.in_adj,
                               fwd ? (mine ? o.off_out : S.off_out[q]) : (mine ? o.off_in : S.off_in[q]), la, d,
                               ctr) >= 0;
        if (found) return false;
      }
    }
    return true;
  }
  return check_leaf_searched<kC>(G, P, S, grp, p, drive, d, o, ctr);
}

// ---- shared position-0 states: choosing position 1 last ---------------------
//
// With P.defer1 every seed (u, v) of one position-0 image u shares the search
// over positions 2..k-1, which never looks at position 1 (no pattern arc
// joins it to a later position).  A warp extends one image u with position 1
// unset; at each complete assignment M of the other positions it chooses
// position 1 among the group's seed images v: v must not be in M, and in
// induced mode the non-arcs between position 1 and later positions (P.defer)
// must hold.  Positions 0..nmapped-1 are in S.map (S.map[1] = -1); the last
// one or two positions are given: mK at k-1 and, when nmapped == k-2, mL at k-2.

// Is there an arc x -> y (any label)?
template <bool kC>
__device__ __forceinline__ bool arc_exists(const DevGraph &G, int32_t x, int32_t y, Bytes &ctr) {
  int32_t lab;
  if (G.filt_min >= 0) return arc_maybe<kC>(G, x, y, ctr) && arc_find<kC>(G, x, y, &lab, ctr);
  if (kC) ctr += 32;
  const int4 ix = __ldg(&G.vi[HM_AT(G, x, G.n, kChkVertex)]), iy = __ldg(&G.vi[HM_AT(G, y, G.n, kChkVertex)]);
  return arc_lookup<kC>(G, x, y, ix.y, iy.z, &lab, ctr);
}

// Is x among the group's images sorted_seeds[lo, hi).y (ascending)?
__device__ __forceinline__ bool group_has(const int2 *__restrict__ sv, int32_t lo, int32_t hi, int32_t x) {
  while (lo < hi) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    const int32_t y = __ldg(&sv[mid].y);
    if (y < x) lo = mid + 1;
    else if (y > x) hi = mid;
    else return true;
  }
  return false;
}

template <bool kRows, bool kC>
__device__ void expand_position1(const DevGraph &G, const Plan &P, const WarpState &S, const ExtArgs &A,
                                 bool ok, int nmapped, int32_t mL, int32_t mK, int lane,
                                 unsigned long long &task_count, unsigned long long *row_cursor,
                                 int32_t *row_base, unsigned long long row_cap, Bytes &ctr) {
  const int k = P.k;
  const int32_t vlo = S.vlo, vhi = S.vhi;
  if (!kRows && P.ndefer == 0) {
    // monomorphism count: every image of the group not used by M
    unsigned long long add = 0;
    if (ok) {
      int used = group_has(A.sorted_seeds, vlo, vhi, mK) ? 1 : 0;
      if (nmapped == k - 2 && group_has(A.sorted_seeds, vlo, vhi, mL)) ++used;
      for (int i = 0; i < nmapped; ++i)
        if (i != 1 && group_has(A.sorted_seeds, vlo, vhi, S.map[i])) ++used;
      add = (unsigned long long)(vhi - vlo - used);
      if (kC) ctr += 8ull * (nmapped + 1);
    }
    for (int o = 16; o; o >>= 1) add += __shfl_xor_sync(kFull, add, o);
    task_count += add;
    return;
  }
  // every (match M of a lane with ok, image v of the group) pair, 32 pairs per step
  const uint32_t okm = __ballot_sync(kFull, ok);
  const int32_t nv = vhi - vlo;
  const int64_t total = (int64_t)__popc(okm) * nv;
  for (int64_t g0 = 0; g0 < total; g0 += 32) {
    const int64_t g = g0 + lane;
    const bool live = g < total;
    const int j = live ? (int)(g / nv) : 0;         // which ok lane's M
    const int32_t vi = live ? (int32_t)(g - (int64_t)j * nv) : 0;
    const int src = (int)__fns(okm, 0, j + 1);       // lane of the (j+1)-th set bit
    const int32_t cL = __shfl_sync(kFull, mL, src);
    const int32_t cK = __shfl_sync(kFull, mK, src);
    bool good = false;
    int32_t v = -1;
    if (live) {
      v = __ldg(&A.sorted_seeds[vlo + vi].y);
      if (kC) {
        ctr += 8;
        ctr.model += 8;
      }
      good = v != cK && (nmapped == k - 1 || v != cL);
      for (int i = 0; i < nmapped && good; ++i)
        if (S.map[i] == v) good = false;  // injective (S.map[1] = -1)
      for (int jj = 0; jj < P.ndefer && good; ++jj) {
        const Cons cs = P.defer[jj];
        const int32_t fq = cs.q < nmapped ? S.map[cs.q] : (cs.q == k - 1 ? cK : cL);
        const bool fwd = cs.kind == kNotOut;  // the forbidden arc is f(q) -> v
        if (arc_exists<kC>(G, fwd ? fq : v, fwd ? v : fq, ctr)) good = false;
      }
    }
    const uint32_t bal = __ballot_sync(kFull, good);
    const int nm = __popc(bal);
    task_count += nm;
    if (kRows && nm) {
      unsigned long long at = 0;
      if (lane == 0) at = atomicAdd(row_cursor, (unsigned long long)nm);
      at = __shfl_sync(kFull, at, 0);
      if (good) {
        const unsigned long long r = at + __popc(bal & lanemask_lt());
        if (r < row_cap) {
          if (kC) {
            ctr += 4 * k;
            ctr.model += 4 * k;
          }
          int32_t *row = row_base + r * k;
          for (int i = 0; i < k; ++i)
            row[P.orig[i]] = i == 1 ? v : (i < nmapped ? S.map[i] : (i == k - 1 ? cK : cL));
        }
      }
    }
  }
}

// Runs the leaf of every survivor in `m` (bits over adj[base + lane]) that has
// at most kFlatMax leaf candidates; returns the survivors left for the
// ordinary descent.  Adds the matches to task_count and writes their rows.
template <bool kRows, bool kC, bool kShared, bool kSym>
__device__ uint32_t leaf_flatten(const DevGraph &G, const Plan &P, WarpState &S, const ExtArgs &A,
                                 int2 *__restrict__ grp, int L, const int32_t *__restrict__ adj,
                                 int32_t base, uint32_t m, int lane, const uint8_t *root_mask,
                                 unsigned long long &task_count, Ctl *ctl, uint32_t &chunks,
                                 Bytes &ctr) {
  const int p = L + 1;
  const int k = P.k;
  const int npos = P.npos[p];
  // label groups of anchors mapped before depth L are the same for every survivor
  bool dead = false;
  for (int j = 0; j < npos; ++j) {
    const Cons cs = P.cons[p][j];
    if (cs.q == L) continue;
    const int4 dq = S.dir[cs.q];
    const int2 r = cs.kind == kOut ? dir_lookup<kC>(G, G.gdir_out, dq.x, dq.y, cs.lab, P.vlab[p], lane, ctr)
                                   : dir_lookup<kC>(G, G.gdir_in, dq.z, dq.w, cs.lab, P.vlab[p], lane, ctr);
    if (lane == 0) grp[P.gbase[p] + j] = r;
    dead |= r.y == 0;
  }
  if (dead) {
    // an anchor mapped before L has no neighbour the leaf could take: no
    // survivor of depth L, now or in the prefix's later chunks, can match
    if (lane == 0) S.hi[L] = S.lo[L];
    __syncwarp();
    return 0;
  }
  __syncwarp();
  // each survivor lane: its record, its own label groups, its shortest range
  const bool mine = (m >> lane) & 1u;
  LeafOwner o{};
  int32_t drv_j = 0, drv_lo = 0, drv_len = 0, drv_kind = 0;
  int4 probe = make_int4(0, 0, 0, 0);
  if (mine) {
    const int32_t c = __ldg(adj + HM_AT(G, (int64_t)base + lane, G.m, kChkList));
    const int4 vi = __ldg(&G.vi[HM_AT(G, c, G.n, kChkVertex)]);
    const int2 of = __ldg(&G.off[HM_AT(G, c, G.n, kChkVertex)]);
    const int4 vd = __ldg(&G.vdir[HM_AT(G, c, G.n, kChkVertex)]);
    if (kC) ctr += 52;
    o.c = c;
    o.off_out = of.x;
    o.off_in = of.y;
    o.deg_out = vi.y;
    o.deg_in = vi.z;
    int32_t best = INT32_MAX;
    for (int j = 0; j < npos; ++j) {
      const Cons cs = P.cons[p][j];
      int2 r;
      int32_t lo;
      if (cs.q == L) {
        const int4 *dir = cs.kind == kOut ? G.gdir_out : G.gdir_in;
        const int32_t first = cs.kind == kOut ? vd.x : vd.z, cnt = cs.kind == kOut ? vd.y : vd.w;
        r = make_int2(0, 0);
        // entries four at a time (independent loads, one round trip per four)
        bool hit = false;
        for (int32_t e0 = 0; e0 < cnt && !hit; e0 += 4) {
          int4 ent[4];
#pragma unroll
          for (int t = 0; t < 4; ++t)
            ent[t] = e0 + t < cnt ? __ldg(dir + HM_AT(G, (int64_t)first + e0 + t,
                                                     cs.kind == kOut ? G.ndir_out : G.ndir_in,
                                                     cs.kind == kOut ? kChkDirOut : kChkDirIn))
                                  : make_int4(0, 0, 0, 0);
          if (kC) ctr += 16 * (uint64_t)min(4, cnt - e0);
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (!hit && e0 + t < cnt && ent[t].x == cs.lab && ent[t].y == P.vlab[p]) {
              r = make_int2(ent[t].z, ent[t].w - ent[t].z);
              hit = true;
            }
        }
        if (cs.kind == kOut) o.own[0] = r; else o.own[1] = r;
        lo = (cs.kind == kOut ? of.x : of.y) + r.x;
      } else {
        r = grp[P.gbase[p] + j];
        lo = (cs.kind == kOut ? S.off_out[cs.q] : S.off_in[cs.q]) + r.x;
      }
      if (r.y < best) {
        best = r.y;
        drv_j = j;
        drv_lo = lo;
        drv_kind = cs.kind;
      }
    }
    drv_len = best;
    // the first other positive condition: one filter probe per candidate
    // rejects most of them before the general check runs
    for (int j = 0; j < npos; ++j) {
      if (j == drv_j) continue;
      const Cons cs = P.cons[p][j];
      const bool own = cs.q == L;
      const int32_t rlen = own ? (cs.kind == kOut ? o.own[0].y : o.own[1].y) : grp[P.gbase[p] + j].y;
      if (use_filter(G, rlen))
        probe = make_int4(own ? c : S.map[cs.q], 1 | (cs.kind == kOut ? 2 : 0) | (j << 8), cs.lab, rlen);
      break;
    }
  }
  const uint32_t keep = __ballot_sync(kFull, mine && drv_len > kFlatMax);
  const int32_t len = (mine && drv_len <= kFlatMax) ? drv_len : 0;
  int32_t incl = len;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, incl, off);
    if (lane >= off) incl += y;
  }
  const int32_t excl = incl - len;
  const int32_t total = __shfl_sync(kFull, incl, 31);
  S.owners[lane] = o;  // lanes without a survivor own an empty range
  S.owner_drive[lane] = make_int4(drv_j, drv_lo, drv_kind, excl);
  S.owner_probe[lane] = probe;
  __syncwarp();
  if (kC && lane == 0 && total) {
    atomicAdd(&ctl->level_chunks[p], (unsigned long long)((total + 31) / 32));
    atomicAdd(&ctl->level_lanes[p], (unsigned long long)total);
  }
  chunks += (uint32_t)((total + 31) / 32);
  // owner of sweep position g: the first survivor lane whose inclusive prefix exceeds g
  auto owner_of = [&](int32_t g) {
    int32_t lo_l = 0, hi_l = 31;
#pragma unroll
    for (int step = 0; step < 5; ++step) {
      const int32_t mid = (lo_l + hi_l) >> 1;
      const int32_t v = __shfl_sync(kFull, incl, mid);
      if (g < v) hi_l = mid; else lo_l = mid + 1;
    }
    return min(lo_l, 31);
  };
  // candidate at sweep position g of owner ow (-1 past the end)
  auto candidate_at = [&](int32_t g, int ow) {
    if (g >= total) return -1;
    const int4 od = S.owner_drive[ow];
    if (kC) {
      ctr += 4;
      ctr.model += 8;
    }
    return __ldg((od.z == kOut ? G.gout_adj : G.gin_adj) + HM_AT(G, (int64_t)od.y + (g - od.w), G.m, kChkList));
  };
  // the next chunk's owners and candidates are fetched while this chunk is checked
  int ow_next = owner_of(lane);
  int32_t d_next = candidate_at(lane, ow_next);
  for (int32_t chunk = 0; chunk < total; chunk += 32) {
    const int32_t g = chunk + lane;
    const int ow = ow_next;
    const int32_t d = d_next;
    if (chunk + 32 < total) {
      ow_next = owner_of(g + 32);
      d_next = candidate_at(g + 32, ow_next);
    }
    const LeafOwner &oo = S.owners[ow];
    bool ok = false;
    if (g < total) {
      const int4 pr = S.owner_probe[ow];
      ok = true;
      if (pr.y & 1) {
        const bool fwd = pr.y & 2;
        if (kC) ctr.model += search_bytes(pr.w);
        ok = arc_maybe_l<kC>(G, fwd ? pr.x : d, fwd ? d : pr.x, pr.z, ctr);
      }
      if (ok)
        ok = check_leaf<kC, kSym>(G, P, S, grp, p, S.owner_drive[ow].x, (pr.y & 1) ? (pr.y >> 8) : -1, d,
                                  oo, root_mask, ctr);
    }
    if (kShared) {
      expand_position1<kRows, kC>(G, P, S, A, ok, L, oo.c, d, lane, task_count, S.row_cursor, S.row_base,
                                  S.row_cap, ctr);
      continue;
    }
    const uint32_t bal = __ballot_sync(kFull, ok);
    const int nm = __popc(bal) * (kSym ? P.naut : 1);
    task_count += nm;
    if (kRows && nm) {
      unsigned long long at = 0;
      if (lane == 0) at = atomicAdd(S.row_cursor, (unsigned long long)nm);
      at = __shfl_sync(kFull, at, 0);
      if (ok) {
        if (!kSym || P.naut == 1) {
          const unsigned long long r = at + __popc(bal & lanemask_lt());
          if (r < S.row_cap) {
            if (kC) {
              ctr += 4 * k;
              ctr.model += 4 * k;
            }
            int32_t *row = S.row_base + r * k;
            for (int i = 0; i < L; ++i) row[P.orig[i]] = S.map[i];
            row[P.orig[L]] = oo.c;
            row[P.orig[p]] = d;
          }
        } else {
          if (kC) {
            ctr += 4ull * k * P.naut;
            ctr.model += 4ull * k * P.naut;
          }
          write_match_rows(P, S.row_base, at + (unsigned long long)__popc(bal & lanemask_lt()) * P.naut,
                           S.row_cap, S.map, L, oo.c, d);
        }
      }
    }
  }
  __syncwarp();  // every lane is done with S.owners before the next sweep rewrites it
  return keep;
}

// ---- bounded lock-free queue (Vyukov-style sequence numbers) --------------

__device__ __noinline__ bool q_push(const ExtArgs &A, WarpState &S, int lane) {
  long long pos = -1;
  if (lane == 0) {
    atomic_u64 tail(A.ctl->tail);
    unsigned long long p = tail.load(cuda::memory_order_relaxed);
    for (int it = 0; it < 64; ++it) {
      atomic_u64 seq(A.qseq[p & (kQueueCap - 1)]);
      unsigned long long sq = seq.load(cuda::memory_order_acquire);
      long long dif = (long long)sq - (long long)p;
      if (dif == 0) {
        if (tail.compare_exchange_strong(p, p + 1, cuda::memory_order_relaxed)) {
          pos = (long long)p;
          break;
        }
      } else if (dif < 0) {
        break;  // full
      } else {
        p = tail.load(cuda::memory_order_relaxed);
      }
    }
  }
  pos = __shfl_sync(kFull, pos, 0);
  if (pos < 0) return false;
  Task *dst = A.qbuf + (pos & (kQueueCap - 1));
  if (lane < kTaskWords) reinterpret_cast<int32_t *>(dst)[lane] = reinterpret_cast<const int32_t *>(&S.stage)[lane];
  __threadfence();
  __syncwarp();
  if (lane == 0) {
    atomic_u64 seq(A.qseq[pos & (kQueueCap - 1)]);
    seq.store((unsigned long long)pos + 1, cuda::memory_order_release);
  }
  return true;
}

__device__ __noinline__ bool q_pop(const ExtArgs &A, WarpState &S, int lane) {
  long long pos = -1;
  if (lane == 0) {
    atomic_u64 head(A.ctl->head);
    unsigned long long p = head.load(cuda::memory_order_relaxed);
    for (int it = 0; it < 64; ++it) {
      atomic_u64 seq(A.qseq[p & (kQueueCap - 1)]);
      unsigned long long sq = seq.load(cuda::memory_order_acquire);
      long long dif = (long long)sq - (long long)(p + 1);
      if (dif == 0) {
        if (head.compare_exchange_strong(p, p + 1, cuda::memory_order_relaxed)) {
          pos = (long long)p;
          break;
        }
      } else if (dif < 0) {
        break;  // empty (or the producer has not published yet)
      } else {
        p = head.load(cuda::memory_order_relaxed);
      }
    }
    if (pos >= 0) __threadfence();
  }
  pos = __shfl_sync(kFull, pos, 0);
  __syncwarp();
  if (pos < 0) return false;
  const Task *src = A.qbuf + (pos & (kQueueCap - 1));
  if (lane < kTaskWords)
    reinterpret_cast<int32_t *>(&S.stage)[lane] = ((const volatile int32_t *)src)[lane];
  __threadfence();
  __syncwarp();
  if (lane == 0) {
    atomic_u64 seq(A.qseq[pos & (kQueueCap - 1)]);
    seq.store((unsigned long long)pos + kQueueCap, cuda::memory_order_release);
  }
  return true;
}

__device__ __forceinline__ bool queue_maybe_nonempty(const ExtArgs &A) {
  atomic_u64 head(A.ctl->head), tail(A.ctl->tail);
  return tail.load(cuda::memory_order_acquire) > head.load(cuda::memory_order_acquire);
}

// Split the shallowest unfinished range (or pending chunk) and donate one part.
// The task being run may restrict its first chunk [first_lo, first_lo + 32) at
// depth L0 to the candidates in first_mask; a split of that window hands the
// shifted restriction to the new task (such tasks never extend past the window).
__device__ __noinline__ bool try_donate(const ExtArgs &A, const Plan &P, WarpState &S, int L0, int level,
                           int lane, int32_t first_lo, uint32_t first_mask, int32_t pid) {
  int l = -1, kind = 0;
  for (int d = L0; d <= level; ++d) {
    if (S.hi[d] - S.lo[d] >= A.split_min) { l = d; kind = 0; break; }
    if (d < level && __popc(S.mask[d]) >= 2) { l = d; kind = 1; break; }
  }
  if (l < 0) return false;
  if (lane == 0) {
    Task &t = S.stage;
    t.depth = l;
    t.drive = S.drive[l];
    t.pid = pid;
    t.vlo = S.vlo;
    t.vhi = S.vhi;
    for (int i = 0; i < kMaxK; ++i) t.map[i] = i < l ? S.map[i] : -1;
    if (kind == 0) {
      const int32_t mid = S.lo[l] + ((S.hi[l] - S.lo[l]) >> 1);
      t.lo = mid;
      t.hi = S.hi[l];
      t.pmask = kFull;
      if (l == L0 && first_mask != kFull && mid >= first_lo && mid < first_lo + 32)
        t.pmask = first_mask >> (mid - first_lo);
    } else {
      uint32_t m = S.mask[l];
      int keep = __popc(m) >> 1;
      uint32_t mine = 0;
      for (int i = 0; i < keep; ++i) {
        uint32_t low = m & (0u - m);
        mine |= low;
        m ^= low;
      }
      t.lo = S.base[l];
      t.hi = S.base[l] + 32;
      t.pmask = m;  // the upper half goes away
      S.mask[l] = mine;
    }
  }
  __syncwarp();
  bool pushed = q_push(A, S, lane);
  if (lane == 0) {
    if (pushed) {
      if (kind == 0) S.hi[l] = S.stage.lo;
      atomicAdd(&A.ctl->donated, 1ull);
    } else if (kind == 1) {
      S.mask[l] |= S.stage.pmask;  // could not donate: keep the work
    }
  }
  __syncwarp();
  return pushed;
}

// An idle warp advertises itself and waits, with backoff, for a donated task
// or for global quiescence, every wait bounded by the call's deadline.
// Returns true with a task installed in S.stage, false when the call is over.
__device__ __noinline__ bool idle_wait(const ExtArgs &A, WarpState &S, int lane) {
  if (lane == 0) {
    atomicAdd(&A.ctl->hungry, 1);
    atomicAdd(&A.ctl->requests, 1);
    atomicSub(&A.ctl->active, 1);
  }
  unsigned ns = 64;
  for (;;) {
    int quit = 0;
    if (lane == 0) {
      if (ld_volatile(&A.ctl->status) != kStatOk) quit = 1;
      else if (globaltimer_ns() > S.deadline) {
        atomicCAS(&A.ctl->status, kStatOk, kStatBudget);
        quit = 1;
      } else {
        __threadfence();
        int32_t act = ld_volatile(&A.ctl->active);
        __threadfence();
        if (act == 0 && !queue_maybe_nonempty(A)) quit = 1;
      }
      if (!quit && queue_maybe_nonempty(A)) {
        atomicAdd(&A.ctl->active, 1);
        quit = 2;  // try to take it
      }
    }
    quit = __shfl_sync(kFull, quit, 0);
    if (quit == 1) {
      if (lane == 0) atomicSub(&A.ctl->hungry, 1);
      return false;
    }
    if (quit == 2) {
      if (q_pop(A, S, lane)) {
        if (lane == 0) atomicSub(&A.ctl->hungry, 1);
        return true;
      }
      if (lane == 0) atomicSub(&A.ctl->active, 1);
    }
    __nanosleep(ns);
    ns = min(ns * 2, 4096u);
  }
}

// Every 64 chunks: report them, and stop when the call's status is no longer
// ok, its deadline has passed or its chunk budget is spent.  Warp-uniform.
__device__ __noinline__ bool budget_check(const ExtArgs &A, WarpState &S, int lane, uint32_t my_chunks) {
  int halt = 0;
  if (lane == 0) {
    // the status word read here was requested at the previous check, so its
    // latency is hidden
    const unsigned long long add = (uint32_t)(my_chunks - S.chunks_flushed);  // modulo 2^32
    S.chunks_flushed = my_chunks;
    const int32_t status = S.status_seen;
    S.status_seen = ld_volatile(&A.ctl->status);
    if (status != kStatOk) halt = 1;
    else if (globaltimer_ns() > S.deadline) {
      atomicCAS(&A.ctl->status, kStatOk, kStatBudget);
      halt = 1;
    } else if (A.max_chunks) {
      unsigned long long tot = atomicAdd(&A.ctl->chunks, add) + add;
      if (tot > A.max_chunks) {
        atomicCAS(&A.ctl->status, kStatOk, kStatBudget);
        halt = 1;
      }
    } else {
      atomicAdd(&A.ctl->chunks, add);
    }
  }
  return __shfl_sync(kFull, halt, 0) != 0;
}

// Every poll_mask+1 chunks: claim one outstanding donation request.  The
// request count used is the one read at the previous poll, so the poll does
// not stall the warp.  0: nothing to do; 1: donate; 2: no request claimed.
__device__ __noinline__ int poll_requests(const ExtArgs &A, WarpState &S, int lane) {
  int want = 0;
  if (lane == 0) {
    const int32_t asked = S.requests_seen;
    S.requests_seen = ld_volatile(&A.ctl->requests);
    if (asked > 0) want = atomicSub(&A.ctl->requests, 1) > 0 ? 1 : 2;
  }
  return __shfl_sync(kFull, want, 0);
}

__host__ __device__ constexpr size_t warp_smem_bytes(int ngrp) {
  return (sizeof(WarpState) + sizeof(int2) * (size_t)ngrp + 15) / 16 * 16;
}

template <bool kRows, bool kC, int kMinBlocks, bool kBatch, bool kShared = false, bool kSym = false>
__global__ void __launch_bounds__(kExtThreads, kMinBlocks)
k_extend(const __grid_constant__ DevGraph G, const __grid_constant__ Plan P0,
         const __grid_constant__ ExtArgs A) {
  Bytes ctr;
  uint64_t lanes = 0;
  extern __shared__ __align__(16) unsigned char s_raw[];
  const int lane = threadIdx.x & 31;
  const size_t stride = warp_smem_bytes(kBatch ? A.grp_slots : P0.ngrp);
  WarpState &S = *reinterpret_cast<WarpState *>(s_raw + (threadIdx.x >> 5) * stride);
  int2 *grp = reinterpret_cast<int2 *>(s_raw + (threadIdx.x >> 5) * stride + sizeof(WarpState));
  if (lane == 0) {
    S.deadline = globaltimer_ns() + A.budget_ns;
    S.nseeds = *A.nseeds << A.wps_shift;  // claims: (state, part) pairs
    S.seed_at = S.seed_end = 0;
    S.my_count = 0;
    S.chunks_flushed = 0;
    S.requests_seen = 0;
    S.status_seen = kStatOk;
  }
  __syncwarp();
  uint32_t my_chunks = 0, next_check = 64, next_poll = A.poll_mask + 1u;
  bool seeds_done = false, stop = false;
  if (lane == 0) atomicAdd(&A.ctl->active, 1);

  while (!stop) {
    // ---------------- acquire a task ----------------
    int got = 0;  // 1 seed, 2 donated
    int32_t pid = 0;
    if (!seeds_done) {
      unsigned long long seed_at = S.seed_at, seed_end = S.seed_end;
      if (seed_at >= seed_end) {
        unsigned long long s0 = 0;
        if (lane == 0) s0 = atomicAdd(&A.ctl->seed_next, (unsigned long long)A.seeds_per_fetch);
        seed_at = __shfl_sync(kFull, s0, 0);
        seed_end = min(seed_at + (unsigned long long)A.seeds_per_fetch, S.nseeds);
      }
      const unsigned long long s = seed_at;
      __syncwarp();
      if (lane == 0) {
        S.seed_at = seed_at + 1;
        S.seed_end = seed_end;
      }
      __syncwarp();
      if (s < seed_end) {
        const unsigned long long si = s >> A.wps_shift;  // the depth-2 state of this claim
        if (kShared) {
          // a shared position-0 state: position 1 is chosen at the leaves
          const int4 gr = A.groups[si];
          if (kC && lane == 0) ctr += 16;
          set_mapped<kC>(G, S, 0, gr.x, lane, ctr);
          set_mapped<kC>(G, S, 1, -1, lane, ctr);
          if (lane == 0) {
            S.vlo = gr.y;
            S.vhi = gr.z;
          }
        } else {
          const int2 uv = A.seeds[si];
          if (kBatch) pid = A.seed_pid[si];
          if (kC && lane == 0) {
            ctr += kBatch ? 12 : 8;
            ctr.model += 8;
          }
          set_mapped<kC>(G, S, 0, uv.x, lane, ctr);
          set_mapped<kC>(G, S, 1, uv.y, lane, ctr);
          // symmetry breaking between positions 0 and 1: the seed is kept by
          // the extension, not by the validators, so the injected states stay
          // exactly the validators' output
          const Plan &Ps = kBatch ? A.plans[pid] : P0;
          if (kSym && ((Ps.sym_gt[1] && uv.y <= uv.x) || (Ps.sym_lt[1] && uv.y >= uv.x))) {
            __syncwarp();
            continue;
          }
        }
        __syncwarp();
        got = 1;
      } else {
        seeds_done = true;
      }
    }
    if (!got && q_pop(A, S, lane)) got = 2;
    if (!got) {
      if (!idle_wait(A, S, lane)) {
        stop = true;
        break;
      }
      got = 2;
    }
    if (got == 2 && kBatch) pid = S.stage.pid;
    const Plan &P = kBatch ? A.plans[pid] : P0;
    const int k = P.k;
    if (kRows && lane == 0) {
      S.row_cursor = kBatch ? A.row_cursor + pid : &A.ctl->rows_written;
      S.row_base = kBatch ? A.rows + A.row_off[pid] : A.rows;
      S.row_cap = kBatch ? A.row_cap[pid] : A.cap;
    }
    __syncwarp();
    unsigned long long task_count = 0;
    if (got == 1) {
      const int part = (int)((S.seed_at - 1) & ((1ull << A.wps_shift) - 1));  // this claim's share of the state
      if (kBatch && k == 2) {
        // a two-vertex pattern: the validated seed is the whole match (taken by part 0)
        if (lane == 0 && part == 0) {
          atomicAdd(&A.counts[pid], 1ull);
          if (kRows) {
            const unsigned long long r = atomicAdd(S.row_cursor, 1ull);
            if (r < S.row_cap) {
              S.row_base[r * 2 + P.orig[0]] = S.map[0];
              S.row_base[r * 2 + P.orig[1]] = S.map[1];
            }
          }
        }
        __syncwarp();
        continue;
      }
      setup_level<kC>(G, P, S, grp, 2, lane, false, ctr);
      if (A.wps_shift) {
        // several warps share the state: this one takes part `part` of its
        // depth-2 candidate range
        __syncwarp();
        if (lane == 0) {
          const int64_t lo = S.lo[2], len = (int64_t)S.hi[2] - lo, w = 1ll << A.wps_shift;
          S.lo[2] = (int32_t)(lo + len * part / w);
          S.hi[2] = (int32_t)(lo + len * (part + 1) / w);
        }
      }
    }
    int L0 = 2;
    uint32_t first_mask = kFull;
    int32_t first_lo = -1;
    if (got == 2) {
      // install a donated task
      const int d = S.stage.depth;
      for (int i = 0; i < d; ++i) set_mapped<kC>(G, S, i, S.stage.map[i], lane, ctr);
      if (lane == 0) {
        S.vlo = S.stage.vlo;
        S.vhi = S.stage.vhi;
      }
      __syncwarp();
      setup_level<kC>(G, P, S, grp, d, lane, true, ctr);
      if (lane == 0) {
        S.drive[d] = S.stage.drive;
        S.lo[d] = S.stage.lo;
        S.hi[d] = S.stage.hi;
        S.mask[d] = 0;
      }
      __syncwarp();
      L0 = d;
      first_mask = S.stage.pmask;
      first_lo = S.stage.lo;
    }
    __syncwarp();

    // ---------------- depth-first extension ----------------
    int level = L0;
    while (true) {
      if (S.mask[level] == 0) {
        const int32_t lo = S.lo[level];
        int32_t hi = S.hi[level];
        if (lo >= hi) {
          if (level == L0) break;
          --level;
          continue;
        }
        ++my_chunks;
        if ((int32_t)(my_chunks - next_check) >= 0) {
          next_check = my_chunks + 64;
          if (budget_check(A, S, lane, my_chunks)) { stop = true; break; }
        }
        if ((int32_t)(my_chunks - next_poll) >= 0) {
          next_poll = my_chunks + A.poll_mask + 1u;
          // one donation per idle warp's request
          const int want = poll_requests(A, S, lane);
          if (want) {
            bool gave = false;
            if (want == 1) {
              gave = try_donate(A, P, S, L0, level, lane, first_lo, first_mask, pid);
              hi = S.hi[level];  // a split of this level keeps [lo, mid)
            }
            if (lane == 0 && !gave) atomicAdd(&A.ctl->requests, 1);  // not claimed / nothing to give
          }
        }
        const int drive = S.drive[level];
        const Cons dc = P.cons[level][drive];
        const int32_t *adj = dc.kind == kOut ? G.gout_adj : G.gin_adj;
        uint32_t allow = kFull;
        if (level == L0 && first_mask != kFull && lo >= first_lo && lo < first_lo + 32)
          allow = first_mask >> (lo - first_lo);
        const bool leaf = level == k - 1;
        const int J = P.ncons[level] - 1;  // conditions besides the driving one
        bool ok = false;
        int32_t c = -1;
        uint32_t m;
        int take;
        if (A.pair_mode && J >= 2 && J < 32 && (hi - lo) * J <= 32) {
          // the whole range fits one round of (candidate, condition) pairs:
          // a candidate's searches run side by side instead of one after another
          take = (int)(hi - lo);
          const int ci = lane / J, slot = lane - ci * J;
          bool pass = false;
          if (ci < take && ((allow >> ci) & 1u)) {
            const int32_t cc = __ldg(adj + HM_AT(G, (int64_t)lo + ci, G.m, kChkList));
            if (kC && slot == 0) {
              ctr += 4;
              ctr.model += 8;
              ++lanes;
            }
            pass = check_one<kC, kSym>(G, P, S, grp, level, slot < drive ? slot : slot + 1, cc, slot == 0,
                                 leaf, A.root_mask, ctr);
          }
          const uint32_t bal = __ballot_sync(kFull, pass);
          const uint32_t need = (1u << J) - 1u;
          m = 0;
          for (int i = 0; i < take; ++i)
            if (((bal >> (i * J)) & need) == need) m |= 1u << i;
          if (lane < take && ((m >> lane) & 1u)) {
            ok = true;
            c = __ldg(adj + HM_AT(G, (int64_t)lo + lane, G.m, kChkList));
          }
        } else {
          take = 32;
          const int32_t idx = lo + lane;
          if (idx < hi && ((allow >> lane) & 1u)) {
            c = __ldg(adj + HM_AT(G, idx, G.m, kChkList));
            if (kC) {
              ctr += 4;
              ctr.model += 8;
              ++lanes;
            }
            ok = check_candidate<kC, kSym>(G, P, S, grp, level, drive, c, leaf, A.root_mask, ctr);
          }
          m = __ballot_sync(kFull, ok);
        }
        if (kC && ok) ctr.model += 4;  // the survivor's label
        if (A.lookahead && level <= k - 3 && P.nla[level] && m) {
          // look-ahead on the survivors of an inner depth
          ok = ok && lookahead_ok<kC>(G, P, level, c, ctr);
          m = __ballot_sync(kFull, ok);
        }
        if (lane == 0) S.lo[level] = lo + take;
        if (kC && lane == 0) {
          atomicAdd(&A.ctl->level_chunks[level], 1ull);
          atomicAdd(&A.ctl->level_lanes[level], (unsigned long long)min((int32_t)take, hi - lo));
        }
        if (kShared && leaf) {
          // leaf of a shared position-0 state: choose position 1 for each survivor
          expand_position1<kRows, kC>(G, P, S, A, ok, k - 1, -1, c, lane, task_count, S.row_cursor,
                                      S.row_base, S.row_cap, ctr);
          __syncwarp();
          continue;
        }
        if (leaf) {
          // leaf: every survivor is a match (with its automorphic images)
          const int nm = __popc(m) * (kSym ? P.naut : 1);
          task_count += nm;
          if (kRows && nm) {
            unsigned long long at = 0;
            if (lane == 0) at = atomicAdd(S.row_cursor, (unsigned long long)nm);
            at = __shfl_sync(kFull, at, 0);
            if (ok && (!kSym || P.naut == 1)) {
              const unsigned long long r = at + __popc(m & lanemask_lt());
              if (r < S.row_cap) {
                if (kC) {
                  ctr += 4 * k;
                  ctr.model += 4 * k;
                }
                int32_t *row = S.row_base + r * k;
                for (int i = 0; i < k - 1; ++i) row[P.orig[i]] = S.map[i];
                row[P.orig[k - 1]] = c;
              }
            } else if (ok) {
              if (kC) {
                ctr += 4ull * k * P.naut;
                ctr.model += 4ull * k * P.naut;
              }
              write_match_rows(P, S.row_base, at + (unsigned long long)__popc(m & lanemask_lt()) * P.naut,
                               S.row_cap, S.map, k - 1, c, 0);
            }
          }
          __syncwarp();
          continue;
        }
        uint32_t pending = m;
        if (A.leaf_flatten && level == k - 2 && m)
          pending = leaf_flatten<kRows, kC, kShared, kSym>(G, P, S, A, grp, level, adj, lo, m, lane, A.root_mask,
                                            task_count, A.ctl, my_chunks, ctr);
        if (lane == 0) {
          S.mask[level] = pending;
          S.base[level] = lo;
        }
        __syncwarp();
        continue;
      }
      // descend into the next pending survivor
      const uint32_t m = S.mask[level];
      const int b = __ffs(m) - 1;
      const Cons dc = P.cons[level][S.drive[level]];
      const int32_t *adj = dc.kind == kOut ? G.gout_adj : G.gin_adj;
      const int32_t c = __ldg(adj + HM_AT(G, (int64_t)S.base[level] + b, G.m, kChkList));
      __syncwarp();
      if (lane == 0) S.mask[level] = m & (m - 1);
      if (kC && lane == 0) ctr += 4;
      set_mapped<kC>(G, S, level, c, lane, ctr);
      __syncwarp();
      ++level;
      setup_level<kC>(G, P, S, grp, level, lane, false, ctr);
      __syncwarp();
    }
    if (kBatch) {
      if (lane == 0 && task_count) atomicAdd(&A.counts[pid], task_count);
    } else if (lane == 0) {
      S.my_count += task_count;
    }
  }
  if (lane == 0) {
    if (!stop) atomicSub(&A.ctl->active, 1);
    if (S.my_count) atomicAdd(&A.ctl->count, S.my_count);
    if (my_chunks != S.chunks_flushed)
      atomicAdd(&A.ctl->chunks, (unsigned long long)(uint32_t)(my_chunks - S.chunks_flushed));
  }
  if (kC) {
    for (int o = 16; o; o >>= 1) {
      ctr.req += __shfl_xor_sync(kFull, ctr.req, o);
      ctr.model += __shfl_xor_sync(kFull, ctr.model, o);
      lanes += __shfl_xor_sync(kFull, lanes, o);
    }
    if (lane == 0) {
      atomicAdd(&A.ctl->bytes_extend, (unsigned long long)ctr.req);
      atomicAdd(&A.ctl->bytes_extend_model, (unsigned long long)ctr.model);
      atomicAdd(&A.ctl->lanes, (unsigned long long)lanes);
    }
  }
}

// two-vertex patterns: every seed is a match
__global__ void k_seed_rows(const __grid_constant__ Plan P, const int2 *__restrict__ seeds,
                            const unsigned long long *__restrict__ nseeds, int32_t *__restrict__ rows,
                            unsigned long long cap, Ctl *ctl) {
  const unsigned long long n = *nseeds;
  for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < n;
       s += (unsigned long long)gridDim.x * blockDim.x) {
    if (rows && s < cap) {
      int2 uv = seeds[s];
      rows[s * 2 + P.orig[0]] = uv.x;
      rows[s * 2 + P.orig[1]] = uv.y;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->count = n;
}

__global__ void k_qinit(unsigned long long *seq) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < kQueueCap;
       i += (unsigned long long)gridDim.x * blockDim.x)
    seq[i] = i;
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------

struct Timer {
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaStream_t s;
  bool on;
  Timer(cudaStream_t st, bool enabled) : s(st), on(enabled) {
    if (on) {
      cudaEventCreate(&ev[0]);
      cudaEventCreate(&ev[1]);
      cudaEventRecord(ev[0], s);
    }
  }
  void stop() {
    if (on) cudaEventRecord(ev[1], s);
  }
  // Elapsed time; call only after the stream has been synchronised.
  float ms() {
    float t = 0.f;
    if (on && cudaEventQuery(ev[1]) == cudaSuccess) cudaEventElapsedTime(&t, ev[0], ev[1]);
    return t;
  }
  ~Timer() {
    if (on) {
      cudaEventDestroy(ev[0]);
      cudaEventDestroy(ev[1]);
    }
  }
};

// Stream-ordered temporaries of one call, freed (stream-ordered) when it ends.
struct Scratch {
  cudaStream_t s;
  std::vector<void *> p;
  explicit Scratch(cudaStream_t st) : s(st) { p.reserve(16); }
  cudaError_t get(void **out, size_t bytes) {
    cudaError_t e = cudaMallocAsync(out, bytes ? bytes : 16, s);
    if (e == cudaSuccess) p.push_back(*out);
    return e;
  }
  ~Scratch() {
    for (void *q : p) cudaFreeAsync(q, s);
  }
};

using ExtendKernel = void (*)(DevGraph, Plan, ExtArgs);

// Occupancy variants: resident 256-thread blocks per SM requested from the
// compiler (it caps registers per thread accordingly).
constexpr int kMinBlockChoices[3] = {4, 5, 6};

int min_blocks_slot(int min_blocks) {
  for (int i = 0; i < 3; ++i)
    if (kMinBlockChoices[i] == min_blocks) return i;
  return 0;
}

template <bool R, bool C, bool B, bool S, bool Y>
ExtendKernel extend_kernel_mb(int slot) {
  switch (slot) {
    case 1: return k_extend<R, C, 5, B, S, Y>;
    case 2: return k_extend<R, C, 6, B, S, Y>;
    default: return k_extend<R, C, 4, B, S, Y>;
  }
}

template <bool B, bool S, bool Y>
ExtendKernel extend_kernel_s(bool rows, bool counters, int slot) {
  if (rows)
    return counters ? extend_kernel_mb<true, true, B, S, Y>(slot) : extend_kernel_mb<true, false, B, S, Y>(slot);
  return counters ? extend_kernel_mb<false, true, B, S, Y>(slot) : extend_kernel_mb<false, false, B, S, Y>(slot);
}

// The extension kernel for a launch; `shared` (shared position-0 states)
// exists for single-pattern launches only, and never with symmetry breaking
// (`sym`: some pattern of the launch has a plan with naut > 1).
template <bool B = false>
ExtendKernel extend_kernel(bool rows, bool counters, int slot = 0, bool shared = false, bool sym = false) {
  if constexpr (!B) {
    if (shared) return extend_kernel_s<false, true, false>(rows, counters, slot);
  }
  return sym ? extend_kernel_s<B, false, true>(rows, counters, slot)
             : extend_kernel_s<B, false, false>(rows, counters, slot);
}

// Resident blocks of an extension kernel variant for a dynamic shared-memory size.
template <bool B = false>
int extend_grid(bool rows, bool counters, size_t smem, int slot = 0, bool shared = false, bool sym = false) {
  static std::atomic<int> cache[3][16][64];  // zero-initialised (static storage)
  const int sm = (int)std::min<size_t>(smem / 1024, 63);
  std::atomic<int> &c =
      cache[slot][(sym ? 8 : 0) + (shared ? 4 : 0) + (rows ? 2 : 0) + (counters ? 1 : 0)][sm];
  int v = c.load(std::memory_order_relaxed);
  if (!v) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, extend_kernel<B>(rows, counters, slot, shared, sym), kExtThreads, smem);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    v = std::max(per_sm, 1) * num_sms();
    c.store(v, std::memory_order_relaxed);
  }
  return v;
}

}  // namespace
}  // namespace hm
