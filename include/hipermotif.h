/*
 * hipermotif.h -- C ABI of the GB300 (sm_103a) subgraph-matching library.
 *
 * The library finds every match of a small labelled pattern graph G1 in a
 * large labelled target digraph G2 (Sec. II-A): every injective
 * f : V1 -> V2 with equal vertex labels (Eq. 2), every pattern arc mapped to a
 * target arc with an equal label (Eq. 3), and, in induced mode, no target arc
 * between the images of a pattern non-arc (Eq. 1, "<=>"); monomorphism keeps
 * only "=>".  It follows the HiPerMotif method (Sec. III): the pattern is
 * reordered by degree (Alg. 1); every target arc is tried as the image of the
 * reordered pattern's first arc (positions 0 and 1); vertex and edge
 * validators (Alg. 2, Alg. 3) reject candidates; survivors are injected as
 * depth-2 partial mappings and extended vertex by vertex in parallel (the
 * HiPerMotif algorithm of Sec. III-C).
 *
 * Conventions for every entry point
 *   - Plain pointers and sizes only.  "host" pointers are ordinary CPU
 *     memory; "device" pointers are CUDA global memory on the current device.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is stream-ordered on it; a call that returns a count on
 *     the host synchronises with its own copy of that count, nothing more.
 *   - Every call returns an hm_status and never aborts, traps or exits.  On an
 *     error no output is written unless the entry point says otherwise.
 *   - Vertex ids are int32 in [0, n); labels are arbitrary int32 values;
 *     counts are uint64 (a match is a mapping, so automorphic copies count
 *     separately).  Rows are written in ORIGINAL pattern-vertex order
 *     (f(0), ..., f(k-1)) and returned sorted ascending lexicographically.
 *   - The target must be a simple digraph: no self-loop (u, u) and no
 *     repeated ordered pair (u, v); the loaders reject anything else.
 *   - Objects are created on the device that is current at creation and must
 *     be used with that device current.  hm_graph / hm_pattern objects are
 *     read-only after creation and may be shared by concurrent calls on
 *     different streams.
 */
#ifndef HIPERMOTIF_H
#define HIPERMOTIF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HM_OK = 0,
  HM_ERR_ARG = 1,       /* bad pointer, size, id out of range, bad mode      */
  HM_ERR_SELF_LOOP = 2, /* target or pattern has an arc (u, u)               */
  HM_ERR_DUP_EDGE = 3,  /* target or pattern repeats an ordered pair (u, v)  */
  HM_ERR_PATTERN = 4,   /* pattern k < 2, k > HM_MAX_K, no arc, or not weakly connected */
  HM_ERR_OOM = 5,       /* a device allocation failed                        */
  HM_ERR_CAPACITY = 6,  /* output buffer too small; *count holds the needed rows */
  HM_ERR_BUDGET = 7,    /* the device work budget ran out; results invalid   */
  HM_ERR_CUDA = 8,      /* a CUDA runtime call failed                        */
  HM_ERR_NO_DEVICE = 9  /* no CUDA device is usable                          */
} hm_status;

typedef enum { HM_MONO = 0, HM_INDUCED = 1 } hm_mode;

enum { HM_MAX_K = 20 };

typedef struct hm_graph hm_graph;     /* opaque: device-resident target graph  */
typedef struct hm_pattern hm_pattern; /* opaque: reordered pattern and plans   */

/* Human-readable name of a status (static string, never NULL). */
const char *hm_status_str(hm_status s);

/* ------------------------------------------------------------------------
 * Target graph.
 *
 * hm_load_graph -- builds the device-resident target (the paper's double-
 * index storage, Sec. III-D: CSR plus the per-arc source array, and
 * contiguous attribute arrays) from an arc list.
 *   n           vertices (>= 0); m arcs (>= 0).
 *   src, dst    int32[m] arc endpoints; vlab int32[n]; elab int32[m].
 *   device_ptrs 0: the four arrays are host memory; 1: device memory.
 *   stream      stream for the build (see conventions).
 *   out         receives the new graph; the caller frees it with hm_free_graph.
 * Layout built: out-lists (CSR) sorted by (src, dst) and in-lists (CSC) sorted
 * by (dst, src), each with its arc labels, the CSR-order source array, and per
 * vertex {label, out-degree, in-degree} and {out-offset, in-offset}; copies
 * of both lists grouped by (arc label, neighbour label) with a directory; an
 * arc filter (split-block Bloom filter keyed by (u, v) and (u, v, label), 32
 * bits per arc) and an arc hash table (32 bytes per arc) that replace the
 * paper's O(log d) edge-attribute lookup by one or two cache-sector reads.
 * Device memory: 64 bytes per arc, 16 per directory entry (at most 2 per arc)
 * and 40 per vertex (hm_graph_info reports the total).
 * The input arrays are copied; the caller keeps ownership.  m must be below
 * 2^31.  Errors: HM_ERR_ARG (id out of range, n or m negative, m >= 2^31,
 * NULL array),
 * HM_ERR_SELF_LOOP, HM_ERR_DUP_EDGE, HM_ERR_OOM, HM_ERR_CUDA.  Synchronises
 * `stream` before returning.
 * ------------------------------------------------------------------------ */
hm_status hm_load_graph(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                        const int32_t *vlab, const int32_t *elab, int device_ptrs,
                        void *stream, hm_graph **out);

void hm_free_graph(hm_graph *g);

/* hm_load_graph_props -- hm_load_graph with several int32 properties per
 * vertex and per arc.  checkAttributes of the validators compares every
 * property (Sec. III-B; arbitrary numbers of properties, Sec. III-D): two
 * vertices (arcs) have equal labels exactly when all their properties are
 * equal.  Each distinct property tuple is given its rank in the sorted list of
 * distinct tuples as its label, the graph is built on those labels, and the
 * sorted tuple tables are kept with the graph (host memory) for
 * hm_load_pattern_props.
 *   nvp, nep    properties per vertex / per arc, 1..64.
 *   vprops      HOST int32[n * nvp], row-major (vertex v's tuple at v * nvp).
 *   eprops      HOST int32[m * nep], row-major, parallel to src/dst (HOST).
 * Errors as hm_load_graph. */
hm_status hm_load_graph_props(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                              int32_t nvp, const int32_t *vprops, int32_t nep,
                              const int32_t *eprops, void *stream, hm_graph **out);

/* hm_load_pattern_props -- a pattern for a graph loaded with
 * hm_load_graph_props: its vertices carry g's nvp properties (HOST int32[k *
 * nvp]) and its arcs g's nep properties (HOST int32[mp * nep]).  A tuple g
 * does not have gets label -1, which no target vertex or arc carries.
 * Otherwise as hm_load_pattern (Alg. 1, validation).  HM_ERR_ARG if g was not
 * loaded with properties. */
hm_status hm_load_pattern_props(const hm_graph *g, int32_t k, int32_t mp, const int32_t *src,
                                const int32_t *dst, const int32_t *vprops,
                                const int32_t *eprops, hm_pattern **out);

/* Sizes of a loaded graph (host outputs; any may be NULL). */
hm_status hm_graph_info(const hm_graph *g, int32_t *n, int64_t *m, size_t *device_bytes);

/* Bounds-checked builds (the library compiled with HM_CHECK=1,
 * libhipermotif_check.so): every index a kernel forms into one of g's arrays
 * (vertex records, list positions, directory entries, filter blocks, hash
 * buckets) is tested against that array's length before the access; the
 * first index out of range is recorded per graph and replaced by 0, so the
 * kernel reads inside the array and runs on (no fault, no trap).  This call
 * copies the record to *violation (HOST) and clears it: 0 = none; otherwise
 * bit 63 set, bits 48..55 the site (1 vertex record, 2 / 3 out / in directory
 * entry, 4 list position, 5 filter block, 6 hash bucket) and bits 0..47 the
 * index.  Synchronises the device.  In the default build the checks are not
 * compiled in: *violation = 0 and HM_ERR_ARG. */
hm_status hm_check_status(const hm_graph *g, uint64_t *violation);

/* Copy the built adjacency back to HOST buffers (for inspection and tests):
 * out_off/in_off int64[n+1]; out_adj/out_elab/in_adj/in_elab int32[m].
 * Any pointer may be NULL to skip that array.  Synchronous. */
hm_status hm_graph_export(const hm_graph *g, int64_t *out_off, int32_t *out_adj,
                          int32_t *out_elab, int64_t *in_off, int32_t *in_adj,
                          int32_t *in_elab);

/* Copy the label-grouped adjacency back to HOST buffers (inspection, tests).
 * Each vertex's out-list (in-list) is also kept ordered by (arc label,
 * neighbour label, neighbour id); one directory entry per such group.
 *   gout_adj, gin_adj  int32[m]: the grouped lists (same offsets as the plain ones).
 *   vdir               int32[4n]: per vertex {first out entry, out entries,
 *                      first in entry, in entries}.
 *   gdir_out, gdir_in  int32[4 * entries]: {arc label, neighbour label, first,
 *                      end}, first/end relative to the vertex's list start.
 *   ndir               int64[2]: number of out and in entries.
 * Any pointer may be NULL.  Synchronous. */
hm_status hm_graph_export_groups(const hm_graph *g, int32_t *gout_adj, int32_t *gin_adj,
                                 int32_t *vdir, int32_t *gdir_out, int32_t *gdir_in,
                                 int64_t *ndir);

/* ------------------------------------------------------------------------
 * Pattern graph.
 *
 * hm_load_pattern -- validates the pattern and runs Alg. 1 (Structural
 * Reordering, Sec. III-A): sigma(v) = (totaldeg, outdeg); the sigma-argmax
 * takes position 0; each next position takes the sigma-argmax among the
 * unplaced out-neighbours of the last placed vertex, else among all unplaced
 * vertices.  Readings where the paper is silent: ties go to the lowest
 * original id; degrees are static; and if the fallback pick has no arc to a
 * placed vertex, the sigma-argmax among unplaced vertices that do have one is
 * taken instead, so every position after 0 is anchored.  It then builds the
 * per-position plans used by the kernels for both modes.
 *   k     pattern vertices, 2 <= k <= HM_MAX_K;  mp  pattern arcs (>= 1).
 *   src, dst int32[mp], vlab int32[k], elab int32[mp]: HOST memory.
 *   out   receives the pattern; free with hm_free_pattern.  Host-only: needs no GPU.
 * Errors: HM_ERR_ARG, HM_ERR_SELF_LOOP, HM_ERR_DUP_EDGE, HM_ERR_PATTERN.
 * ------------------------------------------------------------------------ */
hm_status hm_load_pattern(int32_t k, int32_t mp, const int32_t *src, const int32_t *dst,
                          const int32_t *vlab, const int32_t *elab, hm_pattern **out);

/* hm_load_pattern_ordered -- as hm_load_pattern, but the visiting order is
 * the caller's instead of Alg. 1's (for ablations of the reordering,
 * Sec. IV-C): order (HOST int32[k]) lists the original vertex at each
 * position.  It must be a permutation (else HM_ERR_ARG) in which every
 * position after the first has an arc, in either direction, to an earlier
 * position (else HM_ERR_PATTERN).  Results never depend on the order. */
hm_status hm_load_pattern_ordered(int32_t k, int32_t mp, const int32_t *src, const int32_t *dst,
                                  const int32_t *vlab, const int32_t *elab, const int32_t *order,
                                  hm_pattern **out);

void hm_free_pattern(hm_pattern *p);

/* order_out (host int32[k]) receives Alg. 1's result: order_out[i] is the
 * original pattern vertex placed at position i.  Host-only. */
hm_status hm_pattern_order(const hm_pattern *p, int32_t *order_out);

/* hm_pattern_automorphisms -- the number of label-preserving automorphisms of
 * the pattern that its search uses for symmetry breaking (the matches of
 * Sec. II-A come in orbits of this size; see hm_tuning.symmetry): the order of
 * the automorphism group when it is between 2 and 64, else 1 (the group is
 * trivial, too large, or the pattern has two vertices).  Host only.
 *   count HOST output. */
hm_status hm_pattern_automorphisms(const hm_pattern *p, int32_t *count);

/* ------------------------------------------------------------------------
 * Matching.
 *
 * hm_count_matches -- number of matches of p in g (Sec. II-A), computed by
 * the HiPerMotif hot path (Sec. III-B, III-C): edge scan with the vertex and
 * edge validators, state injection at depth 2, parallel extension.
 *   mode   HM_MONO or HM_INDUCED.
 *   count  HOST uint64 output.
 * Errors: HM_ERR_ARG, HM_ERR_BUDGET (count invalid; the library stays
 * usable), HM_ERR_OOM, HM_ERR_CUDA.  Synchronises with its own count copy.
 * ------------------------------------------------------------------------ */
hm_status hm_count_matches(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                           uint64_t *count, void *stream);

/* hm_enumerate_matches -- every match as a row of k int32 (original pattern
 * vertex order), sorted ascending lexicographically, written to rows_dev.
 *   rows_dev  DEVICE int32[cap * k], owned by the caller (may be NULL if cap == 0).
 *   cap       rows available.
 *   count     HOST uint64 output: the number of matches.
 * If count > cap the call returns HM_ERR_CAPACITY with *count set and the
 * content of rows_dev unspecified (call again with cap >= *count).  The rows
 * are complete in stream order on `stream` when the call returns.
 * Errors as hm_count_matches, plus HM_ERR_CAPACITY. */
hm_status hm_enumerate_matches(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                               int32_t *rows_dev, uint64_t cap, uint64_t *count, void *stream);

/* hm_count_matches_rooted -- as hm_count_matches, restricted to matches whose
 * image of ORIGINAL pattern vertex `root` is flagged: root_mask_dev is a DEVICE
 * uint8[n] (non-zero = allowed).  Used to split a large count into checkable
 * parts; the union over a partition of V2 is the full count. */
hm_status hm_count_matches_rooted(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                  int32_t root, const uint8_t *root_mask_dev,
                                  uint64_t *count, void *stream);

/* hm_count_matches_part / hm_enumerate_matches_part -- the same computation
 * restricted to the depth-2 states seeded by target arcs of part `part` of
 * `nparts` contiguous ranges of the CSR arc order (the HiPerMotif algorithm's
 * parallel loop over target arcs, Sec. III-C, split into independent pieces).
 * Part i covers arcs [s(i), s(i+1)) with s(i) = floor(m*i/nparts) rounded
 * down to a multiple of 4 and s(nparts) = m.  Every match has exactly one
 * seeding arc, so the parts' counts add up to the full count and their row
 * sets are disjoint with the full row set as their union; each part's rows are
 * sorted.  0 <= part < nparts, else HM_ERR_ARG.  Otherwise as the full calls. */
hm_status hm_count_matches_part(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                int32_t part, int32_t nparts, uint64_t *count, void *stream);
hm_status hm_enumerate_matches_part(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                    int32_t part, int32_t nparts, int32_t *rows_dev, uint64_t cap,
                                    uint64_t *count, void *stream);

/* hm_count_batch / hm_enumerate_batch -- npat patterns against one graph in
 * one pass (the HiPerMotif algorithm of Sec. III-C run for all of them at
 * once): one scan of the target's arcs validates every arc as the seeding arc
 * of every pattern whose signature (arc label, source label, target label) it
 * carries, and one persistent extension launch serves the depth-2 states of
 * all patterns.  Each result equals the pattern's own hm_count_matches /
 * hm_enumerate_matches result.
 *   patterns  HOST array of npat pattern handles (repeats allowed).
 *   modes     HOST int32[npat], HM_MONO or HM_INDUCED per pattern.
 *   counts    HOST uint64[npat] output, filled on HM_OK and on HM_ERR_CAPACITY.
 *   rows_dev  DEVICE int32 buffer owned by the caller; pattern i's rows go to
 *             rows_dev[row_offsets[i] .. row_offsets[i+1]) (int32 elements),
 *             i.e. up to (row_offsets[i+1]-row_offsets[i]) / k_i rows, sorted.
 *   row_offsets HOST uint64[npat+1], non-decreasing.
 * If any pattern has more rows than its region holds, HM_ERR_CAPACITY with all
 * counts set (call hm_count_batch first to size the regions).  npat == 0 is a
 * no-op.  Errors otherwise as hm_count_matches. */
hm_status hm_count_batch(const hm_graph *g, const hm_pattern *const *patterns,
                         const int32_t *modes, int32_t npat, uint64_t *counts, void *stream);
hm_status hm_enumerate_batch(const hm_graph *g, const hm_pattern *const *patterns,
                             const int32_t *modes, int32_t npat, int32_t *rows_dev,
                             const uint64_t *row_offsets, uint64_t *counts, void *stream);

/* ------------------------------------------------------------------------
 * Query server over one resident graph (continuous batching).
 *
 * hm_server_create -- starts `nslots` dispatcher slots (host threads, each
 * with its own CUDA stream) serving queries against g, which must outlive the
 * server.  A free slot takes the waiting queries, in arrival order, that the
 * device-memory budget admits, up to max_batch, and runs them as one batch;
 * queries that arrive meanwhile join the next free slot's batch, and batches
 * of different slots overlap on the GPU.  Admission by what a query needs:
 * its seed queues, 24 B per target arc whose labels fit its seeding arc
 * (counted per (source label, arc label, target label) when the server is
 * created), plus 12 MiB per batch for the donation queue and control block;
 * the search stacks live in shared memory.  The head query always runs when
 * nothing else does, even if it alone exceeds the budget.  A batch makes one
 * pass: the rows of each query that wants them go to a region of up to 2^18
 * rows (fewer when the budget is short) and the batched enumeration keeps
 * the sorted rows of every query whose count fits; only a query whose count
 * exceeds its region runs again, at its exact size if the remaining budget
 * holds it, else it gets its count only (rows_dropped = 1).
 *   mem_budget  device bytes for admitted queries and their rows (0 = a
 *               quarter of the device memory free at creation, at most
 *               32 GiB); HM_ERR_ARG if it cannot admit one batch.
 * hm_server_submit -- validates and reorders the pattern (as hm_load_pattern,
 *   HOST arrays), queues it and returns its id at once.  mode HM_MONO or
 *   HM_INDUCED; want_rows 0/1.  Thread-safe.
 * hm_server_poll -- done = 1 once the query has completed (wait = 1 blocks
 *   until then).  When done: *count, *latency_ms (submit to completion, host
 *   clock), *rows_dropped, and *rows / *nrows: HOST rows (nrows x k int32,
 *   sorted) owned by the server until hm_server_release.  Returns the query's
 *   status (HM_OK, or the error its batch met).
 * hm_server_release -- frees a completed query's results.
 * hm_server_stats -- batches launched, queries completed, the largest number
 *   of batches that were in flight at once, queries whose rows were dropped.
 * hm_server_destroy -- serves what is queued, joins the slots, frees all.
 * ------------------------------------------------------------------------ */
typedef struct hm_server hm_server;

hm_status hm_server_create(const hm_graph *g, int32_t nslots, int32_t max_batch,
                           uint64_t mem_budget, hm_server **out);
hm_status hm_server_submit(hm_server *s, int32_t k, int32_t mp, const int32_t *src,
                           const int32_t *dst, const int32_t *vlab, const int32_t *elab,
                           int32_t mode, int32_t want_rows, uint64_t *qid);
hm_status hm_server_poll(hm_server *s, uint64_t qid, int32_t wait, int32_t *done, uint64_t *count,
                         double *latency_ms, int32_t *rows_dropped, const int32_t **rows,
                         uint64_t *nrows);
hm_status hm_server_release(hm_server *s, uint64_t qid);
hm_status hm_server_stats(hm_server *s, uint64_t *batches, uint64_t *completed,
                          uint64_t *max_inflight_batches, uint64_t *rows_dropped);
void hm_server_destroy(hm_server *s);

/* hm_injected_states -- the depth-2 states the edge scan produces: every
 * target arc accepted by the vertex validator (Alg. 2) and the edge
 * validator (Alg. 3) for the reordered arc between positions 0 and 1, as
 * pairs (f(pos0), f(pos1)) in unspecified order.
 *   states_dev DEVICE int32[cap * 2]; count HOST output (total states).
 * Returns HM_ERR_CAPACITY (with *count) if cap is too small. */
hm_status hm_injected_states(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                             int32_t *states_dev, uint64_t cap, uint64_t *count,
                             void *stream);

/* ------------------------------------------------------------------------
 * hm_count_matches_static -- hm_count_matches without any device allocation.
 * The paper has no counterpart: this is an interface for callers that cannot
 * allocate device memory while they match, e.g. a process whose device memory
 * is carved up in advance by another allocator (a framework's caching pool or
 * a hard per-process budget), or a latency-critical loop in which cudaMalloc,
 * which may synchronise the whole device, is not acceptable.
 *   Working memory (control block, donation queue, two seed queues) comes from
 *   one file-scope device array of HM_STATIC_SCRATCH_BYTES (64 MiB).  Every GPU
 *   that loads the library holds that array until the process exits.
 *   The graph may have at most HM_STATIC_MAX_ARCS arcs (one seed slot per
 *   arc in each seed queue); a larger graph is rejected with HM_ERR_CAPACITY
 *   before anything is launched.
 *   The first call on a device looks up the array's device address (with that
 *   device current) and caches it; make that first call before any stream
 *   capture.  The call allocates nothing: no cudaMalloc, no cudaFree, no pool.
 *   Every call copies its control block back and synchronises `stream` before
 *   it returns, so the host waits for the count.
 *   All calls on a device share the array, which keeps the previous call's
 *   contents (the call clears what must start at zero): calls whose work
 *   overlaps on the GPU, e.g. on two streams, race on it -- serialise them.
 *   Otherwise as hm_count_matches (same result, same errors), with one
 *   difference in speed: it does not group depth-2 states by their position-0
 *   image (hm_tuning.share_seeds), because the grouping sorts the states into
 *   temporary buffers that the fixed array has no room for, so a pattern with
 *   a pendant position 1 (e.g. the feed-forward loop plus out-edge) takes the
 *   one-search-per-state path. */
enum { HM_STATIC_SCRATCH_BYTES = 64 << 20, HM_STATIC_MAX_ARCS = 3702528 };

hm_status hm_count_matches_static(const hm_graph *g, const hm_pattern *p, hm_mode mode,
                                  uint64_t *count, void *stream);

/* ------------------------------------------------------------------------
 * Work budget (watchdog).  Every extension kernel stops when either limit is
 * reached and the call returns HM_ERR_BUDGET:
 *   max_ms      wall-clock limit per kernel (0 = default, 120000 ms);
 *   max_chunks  limit on 32-candidate chunks examined per call (0 = none).
 * Process-wide setting; takes effect for calls that start afterwards.
 * ------------------------------------------------------------------------ */
hm_status hm_set_budget(uint64_t max_ms, uint64_t max_chunks);

/* ------------------------------------------------------------------------
 * Launch knobs of the extension kernel (process-wide; read by calls that
 * start afterwards).  None of them changes any result, only speed.
 *   extend_min_blocks  resident 256-thread blocks per SM the kernel is
 *                      compiled for: 4 (default, 64 registers per thread),
 *                      5 or 6 (fewer registers, more warps to hide load
 *                      latency, more register spills).
 *   split_min          a busy warp donates half of a candidate range to idle
 *                      warps only while the range holds at least this many
 *                      candidates (default 64, >= 2).
 *   pair_mode          1: when a whole candidate range fits one round of
 *                      (candidate, condition) pairs (candidates x conditions
 *                      <= 32), one lane per pair, so a candidate's searches
 *                      run side by side; 0 (default): one lane per candidate,
 *                      conditions in turn with early exit.
 *   seeds_per_fetch    depth-2 states a warp claims from the seed queue at
 *                      once (default 1, at most 1024).
 *   poll_every         a busy warp looks for idle warps' donation requests
 *                      every poll_every candidate chunks (a power of two,
 *                      1..65536, default 128); each request is claimed by
 *                      exactly one busy warp.
 *   leaf_flatten       1 (default): at the last inner depth, the survivors of
 *                      a chunk look up their leaf ranges side by side and the
 *                      ranges are swept together in full 32-lane chunks
 *                      (survivors with more than 2048 leaf candidates take the
 *                      ordinary path); -1: one survivor at a time.
 *   arc_filter         a membership test ("is (x, y) an arc with label l?",
 *                      "is there no arc?") over a list of more than this many
 *                      sorted entries probes the graph's arc filter (a Bloom
 *                      filter whose "no" is exact) and, on "maybe", its arc
 *                      hash table, instead of a binary search (default 1;
 *                      -1: always binary search).
 *   share_seeds        1 (default): when no later pattern position has an arc
 *                      to position 1, single-pattern calls group the injected
 *                      depth-2 states by their position-0 image, search the
 *                      other positions once per group and choose position 1
 *                      last from the group's seeds, checking the induced
 *                      non-arcs to position 1 there (same result set, far
 *                      less work when hubs carry many seeds); induced calls
 *                      split an image's seeds into groups of at most 32, so
 *                      each group's warp checks few (match, seed) pairs; -1:
 *                      one search per depth-2 state.
 *   symmetry           1 (default): a pattern with a non-trivial group of
 *                      label-preserving automorphisms (at most 64 of them)
 *                      is searched for one map per orbit -- order
 *                      constraints between symmetric positions, chosen by
 *                      orbits and stabilisers -- and each map found is
 *                      emitted with its automorphic images (same count and
 *                      rows; a pattern with two automorphisms takes about
 *                      half the search).  Not used for rooted counts, for
 *                      two-vertex patterns or with shared position-0
 *                      states.  -1: every map is searched for itself.
 *   warps_per_state    1, 2 or 4: warps that share one depth-2 state.
 *                      Each claim from the state queue is a (state, part)
 *                      pair; the warp takes that part of the state's first
 *                      extension range (contiguous equal slices), so a
 *                      hub's state starts on several warps at once instead
 *                      of waiting for donations.  0 (default): automatic --
 *                      4 for shared position-0 states (share_seeds), 1
 *                      otherwise.
 *   lookahead          1: at every inner depth before the last two, a
 *                      candidate must have, for each class (direction, arc
 *                      label, neighbour label) of the pattern arcs from its
 *                      position to later ones, at least as many neighbours
 *                      as those later positions (a labelled form of VF2's
 *                      terminal-set look-ahead; sound, so results are
 *                      unchanged); -1 (default): off.
 * A zero field takes its default.  HM_ERR_ARG for any other value.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t extend_min_blocks;
  int32_t split_min;
  int32_t pair_mode;
  int32_t seeds_per_fetch;
  int32_t poll_every;
  int32_t leaf_flatten;
  int32_t arc_filter;
  int32_t share_seeds;
  int32_t symmetry;
  int32_t warps_per_state;
  int32_t lookahead;
} hm_tuning;

hm_status hm_set_tuning(const hm_tuning *t);
hm_status hm_get_tuning(hm_tuning *t);

/* hm_autotune -- picks the knobs above for a workload: it times the batched
 * count (hm_count_batch) of the given patterns and improves the setting by
 * coordinate descent, one knob at a time over its candidate values (warps
 * per state 1/2/4; queue chunk, i.e. states claimed at once, 1..64; the
 * intersection strategy arc_filter: filter probes, binary search in sorted
 * lists of up to 16 entries, or binary search always; blocks per SM 4/5/6;
 * split threshold 16..1024; poll interval 32/128/512; pair mode; leaf
 * flattening), keeping a change only when it is more than 1 % faster (best of
 * two runs each), until a pass changes nothing or budget_ms of wall time is
 * spent (0 = no limit).  It installs the fastest setting with hm_set_tuning
 * and returns it in *best (its time in *best_ms, may be NULL).  Every run's
 * counts are compared with a reference run's; a difference (which no knob can
 * cause) restores the previous setting and returns HM_ERR_CUDA.  Synchronous. */
hm_status hm_autotune(const hm_graph *g, const hm_pattern *const *patterns, const int32_t *modes,
                      int32_t npat, uint32_t budget_ms, hm_tuning *best, float *best_ms,
                      void *stream);

/* hm_autotune_cached -- hm_autotune with a cache file (host path; NULL or ""
 * = none).  The key is a fingerprint of the graph (its sizes and a strided
 * sample of its sorted arc arrays) and of the workload (how many patterns of
 * each size and mode).  A setting stored under the key is installed without
 * timing (*from_cache = 1, *best_ms = the time stored with it); otherwise the
 * tuner runs and appends its choice to the file as one text line
 * "<key> name=value ... ms=<time>".  from_cache may be NULL. */
hm_status hm_autotune_cached(const hm_graph *g, const hm_pattern *const *patterns,
                             const int32_t *modes, int32_t npat, uint32_t budget_ms,
                             const char *cache_path, hm_tuning *best, float *best_ms,
                             int32_t *from_cache, void *stream);

/* ------------------------------------------------------------------------
 * Statistics of the calling thread's last matching call (host struct).
 * When timing is enabled (hm_set_timing(1)), each kernel launch is bracketed
 * by CUDA events on the call's stream and its duration is reported here.
 * ------------------------------------------------------------------------ */
typedef struct {
  uint64_t seeds_scanned;   /* target arcs scanned by the edge kernel       */
  uint64_t states_injected; /* depth-2 states after both validators         */
  uint64_t tasks_donated;   /* work items split off for idle warps          */
  uint64_t chunks;          /* 32-candidate chunks examined                 */
  uint64_t matches;         /* the count of the call                        */
  float ms_edge_scan;       /* edge scan + validators                       */
  float ms_overlap;         /* neighbour-overlap part of the edge validator,
                             * plus the seed grouping of shared position-0
                             * states (share_seeds)                         */
  float ms_extend;          /* persistent extension kernel                  */
  float ms_sort;            /* row sort (enumerate only)                    */
  int32_t extend_grid;      /* blocks of the extension launch               */
  int32_t extend_block;     /* threads per block                            */
  uint32_t kernel_launches; /* kernels the call launched                    */
  uint32_t pad;
  /* bytes each kernel's accesses requested, at the granularity it reads
   * them (a 32-byte filter block per probe, a 16-byte vertex record, ...);
   * filled only while counters are enabled */
  uint64_t bytes_edge_scan;
  uint64_t bytes_overlap;
  uint64_t bytes_extend;
  uint64_t candidates;      /* candidate vertices examined by the extension */
  uint64_t level_chunks[HM_MAX_K];     /* 32-candidate chunks per depth (counters only) */
  uint64_t level_candidates[HM_MAX_K]; /* candidates per depth (counters only)          */
  /* the same kernels' bytes under the method's cost model (counters only):
   * 12 B per arc scanned and per vertex record gathered, 8 B per candidate
   * read (neighbour + arc label), ceil(log2(d+1)) x 4 B per membership or
   * non-arc test over the shorter list (d entries), 4 B per surviving
   * candidate's label, 4 B per neighbour merged by the overlap test, 8 B per
   * state and 4k B per row written */
  uint64_t model_bytes_edge_scan;
  uint64_t model_bytes_overlap;
  uint64_t model_bytes_extend;
} hm_stats;

hm_status hm_last_stats(hm_stats *out);
hm_status hm_set_timing(int enabled);

/* Enable (1) or disable (0) the algorithmic-byte counters: matching calls then
 * run instrumented kernel variants that tally the bytes they request into
 * hm_stats.  For measurement only -- the instrumented variants are slower. */
hm_status hm_set_counters(int enabled);

#ifdef __cplusplus
}
#endif
#endif /* HIPERMOTIF_H */
