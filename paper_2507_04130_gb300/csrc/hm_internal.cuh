// hm_internal.cuh -- types and device helpers shared by the library's sources.
//
// Layout of a loaded target graph in HBM (all arrays 256-byte aligned):
//   src      int32[m]  source of each arc, CSR order (the per-arc source array
//                      of the double-index storage, Sec. III-D)
//   out_adj  int32[m]  out-neighbours, sorted within each vertex
//   out_elab int32[m]  label of each out-arc, parallel to out_adj
//   in_adj   int32[m]  in-neighbours, sorted within each vertex (CSC)
//   in_elab  int32[m]  label of each in-arc, parallel to in_adj
//   vi       int4[n]   {vertex label, out-degree, in-degree, 0}
//   off      int2[n]   {first out-arc, first in-arc}   (m < 2^31, so 32-bit offsets)
//   afilt    uint4[2*B] arc filter: B = ceil(m/8) blocks of 256 bits holding two
//                      keys per arc, (u, v) and (u, v, label), 16 bits per key
//                      (64 MB for 16M arcs, within the 129 MB L2)
//   ahash    int4[2*H] arc hash table: H = m buckets of two 16-byte slots
//                      {u, v, label, 0} (32 bytes per arc, half the slots used)
// A vertex's label and both degrees arrive in one 16-byte load, its list
// offsets in a second one.  The label-grouped lists and their directory
// (gout_adj, gin_adj, gdir_out, gdir_in, vdir) are described with DevGraph.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "hipermotif.h"

namespace hm {

constexpr int kMaxK = HM_MAX_K;
constexpr int kMaxCons = 2 * (HM_MAX_K - 1);
constexpr int kMaxAut = 64;  // symmetry breaking is used for patterns with at most this many automorphisms
static_assert(kMaxCons <= 64, "condition masks are 64-bit");
constexpr int kWarp = 32;

struct DevGraph {
  int32_t n;
  int64_t m;
  const int32_t *src;
  const int32_t *out_adj;
  const int32_t *out_elab;
  const int32_t *in_adj;
  const int32_t *in_elab;
  const int4 *vi;
  const int2 *off;
  // label-grouped copies of the lists: each vertex's list ordered by
  // (arc label, neighbour label, neighbour id); one directory entry per group
  const int32_t *gout_adj;
  const int32_t *gin_adj;
  const int4 *gdir_out;  // {arc label, neighbour label, first, end} (relative to the list start)
  const int4 *gdir_in;
  const int4 *vdir;      // {first out entry, out entries, first in entry, in entries}
  // split-block Bloom filter over the arcs, keyed by (u, v) and by (u, v,
  // label): a "no" is exact, a "maybe" needs the search.  Searches over more
  // than filt_min entries probe it first (filt_min < 0: never).
  const uint4 *afilt;
  uint32_t afilt_nblk;
  int32_t filt_min;
  // exact arc lookup in one or two 32-byte reads, for what the filter lets through
  const int4 *ahash;
  uint32_t ahash_nbkt;
  // directory lengths, and the violation word of bounds-checked builds (null otherwise)
  int64_t ndir_out, ndir_in;
  unsigned long long *check;
};

// Sites of the bounds checks (HM_CHECK builds): which array an index was meant for.
enum CheckSite : int {
  kChkVertex = 1,   // vi, off, vdir (vertex id < n)
  kChkDirOut = 2,   // gdir_out entry
  kChkDirIn = 3,    // gdir_in entry
  kChkList = 4,     // src, out/in adjacency and labels, grouped lists (position < m)
  kChkFilter = 5,   // arc filter block
  kChkHash = 6,     // arc hash bucket
};

// One pairwise condition between the position being extended (p) and an
// earlier position q, on the candidate c for p:
enum ConsKind : int8_t {
  kOut = 0,     // arc f(q) -> c must exist with label `lab`   (pattern arc q->p)
  kIn = 1,      // arc c -> f(q) must exist with label `lab`   (pattern arc p->q)
  kNotOut = 2,  // no arc f(q) -> c                            (induced, non-arc q->p)
  kNotIn = 3,   // no arc c -> f(q)                            (induced, non-arc p->q)
};

struct Cons {
  int8_t q;
  int8_t kind;
  int16_t pad;
  int32_t lab;
};

// One look-ahead class of a position (see Plan::la).
struct LookClass {
  int8_t kind;   // kOut: arcs f(p) -> later positions; kIn: arcs from them
  int8_t need;   // later positions in the class
  int16_t pad;
  int32_t alab;  // arc label
  int32_t vlab;  // the later positions' vertex label
};

// Per-pattern, per-mode plan, indexed by position after Alg. 1.
struct Plan {
  int32_t k;
  int32_t induced;
  int32_t orig[kMaxK];  // position -> original pattern vertex
  int32_t vlab[kMaxK];  // label required at each position
  int32_t din[kMaxK];   // pattern in-degree at each position
  int32_t dout[kMaxK];  // pattern out-degree at each position
  // the seeding arc between positions 0 and 1
  int32_t seed_rev;     // 0: target arc (a,b) gives f(0)=a, f(1)=b; 1: f(0)=b, f(1)=a
  int32_t seed_lab;     // label of that pattern arc
  int32_t back_req;     // pattern also has 1->0: target arc f(1)->f(0) needed, label back_lab
  int32_t back_lab;
  int32_t back_forbid;  // induced, and the pattern lacks the opposite arc: forbid it in the target
  int32_t ov_need;      // |N(0) & N(1)| in the pattern (neighbour-overlap test)
  int32_t root_pos;     // position whose image must pass a root mask, or -1
  int32_t ncons[kMaxK]; // conditions for position p (positives first)
  int32_t npos[kMaxK];  // how many of them are kOut/kIn
  int32_t gbase[kMaxK]; // first group slot of position p (sum of npos before p)
  int32_t ngrp;         // group slots in total
  // Shared position-0 states: when no later position has a pattern arc to
  // position 1 (defer1), the seeds can be grouped by their position-0 image
  // and position 1 chosen last, from the group's seed list; the induced
  // non-arcs between position 1 and later positions are then checked for
  // each chosen image (defer, with q the later position and the kind read as
  // "f(q) -> v" for kNotOut, "v -> f(q)" for kNotIn).
  int32_t defer1;
  int32_t ndefer;
  Cons cons[kMaxK][kMaxCons];
  Cons defer[kMaxCons];
  // Symmetry breaking.  The matches of a pattern (Sec. II-A, Eqs. 1-3) fall
  // into orbits of |Aut| maps f o s, s an automorphism of the labelled
  // pattern.  The search keeps the one map per orbit that satisfies the order
  // constraints below (f(p) > f(q) for bit q of sym_gt[p], f(p) < f(q) for
  // bit q of sym_lt[p], q < p) and emits it with its |Aut| - 1 images: image
  // s of original vertex v is the vertex at position aut[s][v].  naut = 1:
  // no symmetry breaking (aut[0] maps each vertex to its own position).
  int32_t naut;
  uint32_t sym_gt[kMaxK];
  uint32_t sym_lt[kMaxK];
  int8_t aut[kMaxAut][kMaxK];
  // Look-ahead (a labelled form of VF2's terminal-set rules): a candidate for
  // position p needs, for each class (direction, arc label, neighbour label)
  // of the pattern arcs between p and later positions, at least `need`
  // neighbours of that class -- their images must be distinct.
  int32_t nla[kMaxK];
  LookClass la[kMaxK][kMaxCons];
};

// A plan without symmetry breaking: every map is searched for itself.
inline void strip_symmetry(Plan &P) {
  if (P.naut <= 1) return;
  P.naut = 1;  // aut[0] is the identity
  for (int i = 0; i < kMaxK; ++i) P.sym_gt[i] = P.sym_lt[i] = 0;
}

// Budget / status words shared by all warps of one call.
enum : int32_t { kStatOk = 0, kStatBudget = 1, kStatQueue = 2 };

// Byte tallies of the instrumented kernel variants (hm_set_counters): `req`,
// the bytes the kernel's accesses request at the granularity it reads them
// (a 32-byte filter block per filter probe, a 16-byte vertex record, ...);
// `model`, the method's algorithmic bytes under the survey's cost model: 12 B
// per arc scanned, 12 B per vertex record gathered (label and two degrees),
// 8 B per candidate read from an adjacency list (neighbour and arc label),
// ceil(log2(d+1)) x 4 B per membership or non-arc test (a binary search of
// the shorter list, d entries), 4 B per surviving candidate's label, 4 B per
// neighbour merged by the overlap test, 8 B per state and 4k B per row
// written.  `c += b` adds to req.
struct Bytes {
  uint64_t req = 0, model = 0;
  __host__ __device__ Bytes &operator+=(uint64_t b) {
    req += b;
    return *this;
  }
};

// ceil(log2(d + 1)) x 4: the bytes of a binary search over d sorted entries.
__host__ __device__ __forceinline__ uint64_t search_bytes(int64_t d) {
  uint64_t b = 0;
  while (d > 0) {
    d >>= 1;
    b += 4;
  }
  return b;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

// Is x in the sorted list a[lo, lo+len)?  Returns its index or -1.  Offsets are
// 32-bit (the loader caps m below 2^31).  kCount adds the bytes read to `bytes`.
template <bool kCount>
__device__ __forceinline__ int32_t search_c(const int32_t *__restrict__ a, int32_t lo, int32_t len,
                                            int32_t x, Bytes &bytes) {
  const int32_t end = lo + len;
  while (len > 0) {
    const int32_t half = len >> 1;
    const int32_t v = __ldg(a + lo + half);
    if (kCount) bytes += 4;
    if (v < x) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  if (lo >= end) return -1;
  if (kCount) bytes += 4;
  return __ldg(a + lo) == x ? lo : -1;
}

// ---- arc filter -------------------------------------------------------------
// Every arc (u, v) with label l enters the filter under two keys: the pair
// (u, v) -- "is there an arc at all", for induced non-arcs and the opposite-arc
// test -- and the triple (u, v, l) -- "is there an arc with this label", for
// the pattern's arcs.  A key owns one 256-bit block (eight 32-bit words)
// chosen by the high half of its 64-bit hash and sets one bit in each word;
// bit i sits at the top five bits of the low half times the i-th of eight odd
// constants (a split-block Bloom filter).  The pair hash is the splitmix64
// finalizer (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014); the triple's hash is the pair's xor a
// label-dependent constant.  The eight constants are splitmix64 outputs from
// seed 0x243F6A8885A308D3, made odd.  At 16 bits per key a key that was never
// inserted passes all eight bits with probability about 0.1 %; an inserted key
// always passes.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

struct FilterSlot {
  uint32_t blk;   // block index
  uint32_t bits;  // low half of the key's hash; bit i is at filter_bit(bits, i)
};

__host__ __device__ __forceinline__ FilterSlot filter_slot_of(uint64_t h, uint32_t nblk) {
  FilterSlot f;
  f.blk = (uint32_t)(((h >> 32) * (uint64_t)nblk) >> 32);
  f.bits = (uint32_t)h;
  return f;
}

__host__ __device__ __forceinline__ uint32_t filter_bit(uint32_t bits, int i) {
  const uint32_t salt[8] = {0x2cb0f69fu, 0x94170347u, 0xdd555951u, 0xdbafb151u,
                            0x7e789b2fu, 0xf41e5637u, 0x0959d151u, 0xa97316f1u};
  return (bits * salt[i]) >> 27;
}

__host__ __device__ __forceinline__ uint64_t pair_key(int32_t u, int32_t v) {
  return mix64(((uint64_t)(uint32_t)u << 32) | (uint32_t)v);
}

__host__ __device__ __forceinline__ uint64_t labelled_key(uint64_t pair, int32_t lab) {
  return pair ^ (0x632be59bd9b4e019ull * ((uint64_t)(uint32_t)lab + 1));
}

// ---- bounds checks -------------------------------------------------------------
// Built with HM_CHECK=1 (a separate library, libhipermotif_check.so), every
// index into a graph array passes through HM_AT: one outside [0, n) is
// recorded in *G.check -- bit 63 set, the site in bits 48..55, the index's
// low 48 bits -- if no violation was recorded before, and replaced by 0, so
// the access stays inside the array and the kernel runs on.  The host reads
// and clears the word with hm_check_status.  In the default build HM_AT is
// the index itself.
#ifndef HM_CHECK
#define HM_CHECK 0
#endif
#if HM_CHECK
__device__ __forceinline__ int64_t checked_index(const DevGraph &G, int64_t i, int64_t n, int site) {
  if (i >= 0 && i < n) return i;
  if (G.check)
    atomicCAS(G.check, 0ull,
              (1ull << 63) | ((unsigned long long)(site & 0xff) << 48) | ((unsigned long long)i & 0xffffffffffffull));
  return 0;
}
#define HM_AT(G, i, n, site) ::hm::checked_index((G), (int64_t)(i), (int64_t)(n), (site))
#else
#define HM_AT(G, i, n, site) (i)
#endif

// search_c over one of the graph's lists (every list array has m entries); in
// check builds a span outside [0, m) is recorded and searched as empty
template <bool kCount>
__device__ __forceinline__ int32_t search_g(const DevGraph &G, const int32_t *__restrict__ a, int32_t lo,
                                            int32_t len, int32_t x, Bytes &bytes) {
#if HM_CHECK
  if (len > 0 && (lo < 0 || (int64_t)lo + len > G.m)) {
    checked_index(G, lo < 0 ? (int64_t)lo : (int64_t)lo + len - 1, G.m, kChkList);
    return -1;
  }
#endif
  return search_c<kCount>(a, lo, len, x, bytes);
}

template <bool kCount>
__device__ __forceinline__ bool filter_has(const DevGraph &G, uint64_t h, Bytes &bytes) {
  const FilterSlot f = filter_slot_of(h, G.afilt_nblk);
  const size_t blk = (size_t)HM_AT(G, f.blk, G.afilt_nblk, kChkFilter);
  // the block is one 32-byte sector; its first four words already reject
  // about 98 % of the keys that were never inserted, so the other four are
  // read (from the same sector, now in L1) and tested only when those pass
  const uint4 a = __ldg(G.afilt + 2 * blk);
  if (kCount) bytes += 32;
  const uint32_t x = f.bits;
  const uint32_t t = (a.x >> filter_bit(x, 0)) & (a.y >> filter_bit(x, 1)) & (a.z >> filter_bit(x, 2)) &
                     (a.w >> filter_bit(x, 3));
  if (!(t & 1u)) return false;
  const uint4 b = __ldg(G.afilt + 2 * blk + 1);
  const uint32_t u = (b.x >> filter_bit(x, 4)) & (b.y >> filter_bit(x, 5)) & (b.z >> filter_bit(x, 6)) &
                     (b.w >> filter_bit(x, 7));
  return u & 1u;
}

// false: there is certainly no arc u -> v.  true: there may be.
template <bool kCount>
__device__ __forceinline__ bool arc_maybe(const DevGraph &G, int32_t u, int32_t v, Bytes &bytes) {
  return filter_has<kCount>(G, pair_key(u, v), bytes);
}

// ---- arc hash table -----------------------------------------------------------
// Open addressing over buckets of two 16-byte slots {u, v, label, 0}, one
// 32-byte sector per bucket, with linear probing over buckets from the one the
// pair's hash selects.  Slots fill in order and are never removed, so an empty
// slot (u = -1) ends a probe sequence.  There are as many buckets as arcs
// (half the slots used), so a lookup nearly always reads one sector.
__host__ __device__ __forceinline__ uint32_t hash_bucket(uint64_t pair, uint32_t nbkt) {
  return (uint32_t)(((pair & 0xffffffffull) * (uint64_t)nbkt) >> 32);
}

// Is u -> v an arc?  If so, *lab is its label.
template <bool kCount>
__device__ __forceinline__ bool arc_find(const DevGraph &G, int32_t u, int32_t v, int32_t *lab,
                                         Bytes &bytes) {
  uint32_t b = hash_bucket(pair_key(u, v), G.ahash_nbkt);
  for (uint32_t it = 0; it < G.ahash_nbkt; ++it) {
    const size_t bk = (size_t)HM_AT(G, b, G.ahash_nbkt, kChkHash);
    const int4 s0 = __ldg(G.ahash + 2 * bk);
    const int4 s1 = __ldg(G.ahash + 2 * bk + 1);
    if (kCount) bytes += 32;
    if (s0.x == u && s0.y == v) {
      *lab = s0.z;
      return true;
    }
    if (s1.x == u && s1.y == v) {
      *lab = s1.z;
      return true;
    }
    if (s0.x < 0 || s1.x < 0) return false;
    b = b + 1 == G.ahash_nbkt ? 0 : b + 1;
  }
  return false;
}

// false: there is certainly no arc u -> v with label lab.  true: there may be.
template <bool kCount>
__device__ __forceinline__ bool arc_maybe_l(const DevGraph &G, int32_t u, int32_t v, int32_t lab,
                                            Bytes &bytes) {
  return filter_has<kCount>(G, labelled_key(pair_key(u, v), lab), bytes);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
#endif  // __CUDACC__

}  // namespace hm

// ---------------------------------------------------------------------------
// host-side objects
// ---------------------------------------------------------------------------

namespace hm {
int32_t filter_min();  // current search length above which the arc filter is probed first

// A named range on the host thread's timeline around the launches of one
// phase (NVTX): profilers can select a phase's kernels by it ("ncu --nvtx
// --nvtx-include hm.extend/"); without a tool attached it costs a few ns.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}

struct hm_graph {
  int device;
  int32_t n;
  int64_t m;
  int32_t *src, *out_adj, *out_elab, *in_adj, *in_elab;
  int4 *vi;
  int2 *off;
  int32_t *gout_adj, *gin_adj;
  int4 *gdir_out, *gdir_in, *vdir;
  uint4 *afilt;
  uint32_t afilt_nblk;
  int4 *ahash;
  uint32_t ahash_nbkt;
  int64_t ndir_out, ndir_in;
  unsigned long long *check;  // bounds-checked builds: the violation word (device)
  size_t bytes;
  // multi-property graphs (hm_load_graph_props): the sorted distinct property
  // tuples of vertices and arcs (host, malloc'ed); a label is a tuple's rank
  int32_t nvp, nep;
  int64_t nvtab, netab;
  int32_t *vtab, *etab;
  hm::DevGraph dev() const {
    return hm::DevGraph{n,        m,        src,     out_adj,  out_elab, in_adj,     in_elab,
                        vi,       off,      gout_adj, gin_adj, gdir_out, gdir_in,    vdir,
                        afilt,    afilt_nblk, hm::filter_min(), ahash, ahash_nbkt, ndir_out, ndir_in, check};
  }
};

struct hm_pattern {
  int32_t k, mp;
  int32_t order[HM_MAX_K];
  hm::Plan plan[2];  // [mode]
};

namespace hm {

// Thread-local record of the last call (hm_last_stats).
hm_stats &tls_stats();
bool timing_enabled();
bool counters_enabled();
hm_tuning tuning();  // current process-wide extension knobs (validated)
// log2 of the warps per depth-2 state; 0 (automatic) gives 4 warps to shared
// position-0 states (few, each standing for up to 32 states) and 1 otherwise.
inline int32_t wps_shift(const hm_tuning &t, bool shared = false) {
  if (t.warps_per_state == 0) return shared ? 2 : 0;
  return t.warps_per_state >= 4 ? 2 : t.warps_per_state >= 2 ? 1 : 0;
}
uint64_t budget_ms();
uint64_t budget_chunks();

// Sort rows of `width` int32 words lexicographically by the `nkey` columns
// listed in key_cols (most significant first); every key value must lie in
// [0, 2^bits).  `rows` and `tmp` hold nrows*width words each; the sorted rows
// end in `rows`.  Stable.  Launches on `stream`.
// *launches (if given) receives the number of kernels it launched.
hm_status radix_sort_rows(int32_t *rows, int32_t *tmp, int64_t nrows, int width,
                          const int *key_cols, int nkey, int bits, cudaStream_t stream,
                          int *launches = nullptr);

// As radix_sort_rows, with a bit width (1..32) and an xor mask per key column
// (the xor maps signed values to an unsigned order, e.g. 0x80000000).
hm_status radix_sort_rows_cols(int32_t *rows, int32_t *tmp, int64_t nrows, int width,
                               const int *key_cols, const int *key_bits, const uint32_t *key_xor,
                               int nkey, cudaStream_t stream, int *launches = nullptr);

// out[i] = in[0] + ... + in[i-1] for i in [0, n); values and total below 2^32.
hm_status exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t stream);

// Batched enumeration that keeps what fits (the query server's single pass):
// every count, and for each pattern whose count fits its region [row_offsets[i],
// row_offsets[i+1]) its sorted rows there and fit[i] = 1; fit[i] = 0 otherwise.
hm_status enumerate_batch_fit(const hm_graph *g, const hm_pattern *const *patterns, const int32_t *modes,
                              int32_t npat, int32_t *rows_dev, const uint64_t *row_offsets, uint64_t *counts,
                              uint8_t *fit, cudaStream_t stream);

int bits_for(int64_t n);  // bits needed for values in [0, n)
int num_sms();

}  // namespace hm

#define HM_CUDA_TRY(expr)                                    \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) {                                 \
      (void)cudaGetLastError();                              \
      return e_ == cudaErrorMemoryAllocation ? HM_ERR_OOM    \
                                             : HM_ERR_CUDA;  \
    }                                                        \
  } while (0)
