// hm_graph.cu -- building the device-resident target graph (hm_load_graph).
//
// The paper stores the target in a double-index format: CSR plus an
// arc-to-source array so that both endpoints of an arc are O(1) away, with
// attributes in contiguous arrays and O(log d) edge-attribute lookup in
// sorted adjacency (Sec. III-D).  Here the same storage is built on the GPU
// from an arc list, plus one addition for the extension kernel:
//   1. pack rows (src, dst, label, aux), check ids / self-loops, and find
//      the label ranges                                         (k_pack, k_bounds)
//   2. stable radix sort by (src, dst); split into src / out_adj / out_elab,
//      check repeated pairs, fill out-offsets                    (k_split_out)
//   3. aux = label of dst; stable sort by (src, arc label, dst label): the
//      label-grouped out-lists, and a directory with one entry per
//      (vertex, arc label, neighbour label) group                (k_group_*)
//   4. the same for in-lists, keyed on dst (steps 2-3 mirrored)
//   5. per-vertex records {label, degrees}, {offsets}, {directory spans}
//   6. the arc filter: every arc sets its bits under two keys       (k_filter)
//   7. the arc hash table: every arc claims a slot                  (k_hash)
// The grouped lists let the extension kernel jump straight to the candidates
// whose arc label and vertex label already match (checkAttributes of Alg. 2
// and Alg. 3 applied as a range lookup instead of per candidate).
#include <algorithm>
#include <cstring>
#include <vector>

#include "hm_internal.cuh"

namespace hm {
namespace {

constexpr int kThreads = 256;
constexpr int kW = 4;  // row width: src, dst, arc label, aux

enum : uint32_t { kErrRange = 1, kErrSelf = 2, kErrDup = 4, kErrHash = 8 };

struct Bounds {
  int32_t emin, emax, vmin, vmax;
};

__global__ void k_pack(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                       const int32_t *__restrict__ elab, int64_t m, int32_t n,
                       int32_t *__restrict__ rows, uint32_t *__restrict__ err,
                       Bounds *__restrict__ bnd) {
  int32_t lo = INT32_MAX, hi = INT32_MIN;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = src[e], b = dst[e], l = elab[e];
    uint32_t f = 0;
    if (a < 0 || a >= n || b < 0 || b >= n) f |= kErrRange;
    else if (a == b) f |= kErrSelf;
    if (f) atomicOr(err, f);
    int4 r = make_int4(min(max(a, 0), max(n - 1, 0)), min(max(b, 0), max(n - 1, 0)), l, 0);
    reinterpret_cast<int4 *>(rows)[e] = r;
    lo = min(lo, l);
    hi = max(hi, l);
  }
  atomicMin(&bnd->emin, lo);
  atomicMax(&bnd->emax, hi);
}

__global__ void k_vbounds(const int32_t *__restrict__ vlab, int32_t n, Bounds *__restrict__ bnd) {
  int32_t lo = INT32_MAX, hi = INT32_MIN;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    lo = min(lo, vlab[v]);
    hi = max(hi, vlab[v]);
  }
  atomicMin(&bnd->vmin, lo);
  atomicMax(&bnd->vmax, hi);
}

// off[v] = first row whose key column is >= v, for v in [0, n]; rows sorted by that column.
__device__ __forceinline__ void fill_gap(const int32_t *__restrict__ rows, int col, int64_t e,
                                         int64_t m, int32_t n, int64_t *__restrict__ off) {
  int32_t cur = rows[kW * e + col];
  int32_t prev = e ? rows[kW * (e - 1) + col] : -1;
  for (int32_t v = prev + 1; v <= cur; ++v) off[v] = e;
  if (e == m - 1)
    for (int64_t v = (int64_t)cur + 1; v <= n; ++v) off[v] = m;
}

// Split rows sorted by (key, other): adj = other column, lab = arc label, offsets on key.
__global__ void k_split(const int32_t *__restrict__ rows, int64_t m, int32_t n, int key, int other,
                        int32_t *__restrict__ src_out, int32_t *__restrict__ adj,
                        int32_t *__restrict__ lab, int64_t *__restrict__ off,
                        uint32_t *__restrict__ err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = rows[kW * e + key], b = rows[kW * e + other];
    if (src_out) src_out[e] = a;
    adj[e] = b;
    lab[e] = rows[kW * e + 2];
    if (err && e && rows[kW * (e - 1) + key] == a && rows[kW * (e - 1) + other] == b)
      atomicOr(err, kErrDup);
    fill_gap(rows, key, e, m, n, off);
  }
}

// aux column = label of the neighbour (column `other`)
__global__ void k_set_aux(int32_t *__restrict__ rows, int64_t m, int other,
                          const int32_t *__restrict__ vlab) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    rows[kW * e + 3] = vlab[rows[kW * e + other]];
}

// Rows sorted by (key, arc label, neighbour label, neighbour): grouped list +
// group-start flags (flags[m] = 0 is the scan's sentinel).
__global__ void k_group_flags(const int32_t *__restrict__ rows, int64_t m, int key, int other,
                              int32_t *__restrict__ gadj, uint32_t *__restrict__ flags) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= m;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e == m) {
      flags[m] = 0;
      continue;
    }
    const int32_t *r = rows + kW * e;
    gadj[e] = r[other];
    uint32_t f = 1;
    if (e) {
      const int32_t *q = rows + kW * (e - 1);
      f = (q[key] != r[key] || q[2] != r[2] || q[3] != r[3]) ? 1u : 0u;
    }
    flags[e] = f;
  }
}

// One directory entry per group: {arc label, neighbour label, first, end} relative to the list.
__global__ void k_group_entries(const int32_t *__restrict__ rows, int64_t m, int key,
                                const uint32_t *__restrict__ flags, const uint32_t *__restrict__ idx,
                                const int64_t *__restrict__ off, int4 *__restrict__ dir) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (!flags[e]) continue;
    const int32_t *r = rows + kW * e;
    const int32_t v = r[key];
    const int64_t base = off[v];
    // the group ends at the next group start of the same vertex, or at the list end
    int64_t end = e + 1;
    const int64_t vend = off[v + 1];
    while (end < vend && !flags[end]) ++end;
    dir[idx[e]] = make_int4(r[2], r[3], (int32_t)(e - base), (int32_t)(end - base));
  }
}

__global__ void k_zero_off(int64_t *__restrict__ off, int32_t n) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n;
       v += (int64_t)gridDim.x * blockDim.x)
    off[v] = 0;
}

__global__ void k_vertex(const int32_t *__restrict__ vlab, const int64_t *__restrict__ out_off,
                         const int64_t *__restrict__ in_off, const uint32_t *__restrict__ oidx,
                         const uint32_t *__restrict__ iidx, int32_t n, int4 *__restrict__ vi,
                         int2 *__restrict__ voff, int4 *__restrict__ vdir) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int64_t o0 = out_off[v], o1 = out_off[v + 1], i0 = in_off[v], i1 = in_off[v + 1];
    vi[v] = make_int4(vlab[v], (int32_t)(o1 - o0), (int32_t)(i1 - i0), 0);
    voff[v] = make_int2((int32_t)o0, (int32_t)i0);
    uint32_t os = oidx ? oidx[o0] : 0, oe = oidx ? oidx[o1] : 0;
    uint32_t is = iidx ? iidx[i0] : 0, ie = iidx ? iidx[i1] : 0;
    vdir[v] = make_int4((int32_t)os, (int32_t)(oe - os), (int32_t)is, (int32_t)(ie - is));
  }
}

__device__ __forceinline__ void filter_insert(uint64_t h, uint32_t nblk, uint32_t *__restrict__ words) {
  const FilterSlot f = filter_slot_of(h, nblk);
  uint32_t *w = words + 8 * (size_t)f.blk;
#pragma unroll
  for (int i = 0; i < 8; ++i) atomicOr(w + i, 1u << filter_bit(f.bits, i));
}

__global__ void k_filter(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                         const int32_t *__restrict__ elab, int64_t m, uint32_t nblk,
                         uint32_t *__restrict__ words) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = pair_key(src[e], dst[e]);
    filter_insert(h, nblk, words);
    filter_insert(labelled_key(h, elab[e]), nblk, words);
  }
}

__global__ void k_hash(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                       const int32_t *__restrict__ elab, int64_t m, uint32_t nbkt,
                       int4 *__restrict__ table, uint32_t *__restrict__ err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = src[e], v = dst[e];
    const unsigned long long key = ((unsigned long long)(uint32_t)v << 32) | (uint32_t)u;
    uint32_t b = hash_bucket(pair_key(u, v), nbkt);
    bool placed = false;
    // at most every bucket once: the table has twice as many slots as arcs
    for (uint32_t it = 0; it < nbkt && !placed; ++it) {
      for (int s = 0; s < 2 && !placed; ++s) {
        int4 *slot = table + 2 * (size_t)b + s;
        const unsigned long long old =
            atomicCAS(reinterpret_cast<unsigned long long *>(slot), ~0ull, key);
        if (old == ~0ull) {
          slot->z = elab[e];
          placed = true;
        }
      }
      b = b + 1 == nbkt ? 0 : b + 1;
    }
    if (!placed) atomicOr(err, kErrHash);
  }
}

int grid_for(int64_t work) {
  int64_t g = (work + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)num_sms() * 16));
}

template <typename T>
cudaError_t dmalloc(T **p, int64_t count) {
  return cudaMalloc((void **)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1));
}

void label_key(int32_t lo, int32_t hi, int *bits, uint32_t *xr) {
  if (lo >= 0 && hi < (1 << 24)) {
    *bits = bits_for((int64_t)hi + 1);
    *xr = 0;
  } else {
    *bits = 32;
    *xr = 0x80000000u;  // signed order as unsigned
  }
}

struct Temps {
  cudaStream_t s;
  std::vector<void *> p;
  explicit Temps(cudaStream_t st) : s(st) { p.reserve(16); }
  cudaError_t get(void **out, size_t bytes) {
    cudaError_t e = cudaMallocAsync(out, bytes ? bytes : 16, s);
    if (e == cudaSuccess) p.push_back(*out);
    return e;
  }
  ~Temps() {
    for (void *q : p) cudaFreeAsync(q, s);
  }
};

}  // namespace

void ensure_pool() {
  static thread_local int done_for = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  if (done_for == dev) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done_for = dev;
}

}  // namespace hm

using namespace hm;

namespace {

// Sort `rows` by (key column, arc label, neighbour label) -- rows arrive sorted by
// (key, neighbour), so stability keeps neighbours ascending inside each group --
// then write the grouped list and its directory.
hm_status build_groups(int32_t *rows, int32_t *tmp, int64_t m, int32_t n, int key, int other,
                       const int32_t *vlab, const int64_t *off, int nbits, int be, uint32_t xe,
                       int bv, uint32_t xv, cudaStream_t s, Temps &T, int32_t **gadj, int4 **dir,
                       int64_t *ndir, uint32_t **idx_out) {
  HM_CUDA_TRY(dmalloc(gadj, m));
  k_set_aux<<<grid_for(m), kThreads, 0, s>>>(rows, m, other, vlab);
  const int cols[3] = {key, 2, 3};
  const int bits[3] = {nbits, be, bv};
  const uint32_t xr[3] = {0u, xe, xv};
  hm_status st = radix_sort_rows_cols(rows, tmp, m, kW, cols, bits, xr, 3, s);
  if (st != HM_OK) return st;
  uint32_t *flags, *idx;
  HM_CUDA_TRY(T.get((void **)&flags, sizeof(uint32_t) * (size_t)(m + 1)));
  HM_CUDA_TRY(T.get((void **)&idx, sizeof(uint32_t) * (size_t)(m + 1)));
  k_group_flags<<<grid_for(m + 1), kThreads, 0, s>>>(rows, m, key, other, *gadj, flags);
  st = exclusive_scan_u32(flags, idx, m + 1, s);
  if (st != HM_OK) return st;
  uint32_t total = 0;
  HM_CUDA_TRY(cudaMemcpyAsync(&total, idx + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  HM_CUDA_TRY(cudaStreamSynchronize(s));
  *ndir = total;
  HM_CUDA_TRY(dmalloc(dir, (int64_t)total));
  k_group_entries<<<grid_for(m), kThreads, 0, s>>>(rows, m, key, flags, idx, off, *dir);
  *idx_out = idx;
  return HM_OK;
}

hm_status load_graph_impl(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                          const int32_t *vlab, const int32_t *elab, int device_ptrs,
                          cudaStream_t s, hm_graph *g) {
  Temps T(s);
#if HM_CHECK
  HM_CUDA_TRY(dmalloc(&g->check, 1));  // the bounds checks' violation word
  HM_CUDA_TRY(cudaMemsetAsync(g->check, 0, sizeof(unsigned long long), s));
#endif
  const int32_t *d_src = src, *d_dst = dst, *d_vlab = vlab, *d_elab = elab;
  if (!device_ptrs) {
    int32_t *t;
    HM_CUDA_TRY(T.get((void **)&t, sizeof(int32_t) * (size_t)(3 * m + n + 4)));
    if (m) {
      HM_CUDA_TRY(cudaMemcpyAsync(t, src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
      HM_CUDA_TRY(cudaMemcpyAsync(t + m, dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
      HM_CUDA_TRY(cudaMemcpyAsync(t + 2 * m, elab, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    }
    if (n)
      HM_CUDA_TRY(cudaMemcpyAsync(t + 3 * m, vlab, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    d_src = t;
    d_dst = t + m;
    d_elab = t + 2 * m;
    d_vlab = t + 3 * m;
  }
  int32_t *rows, *tmp;
  int64_t *out_off, *in_off;
  uint32_t *err;
  Bounds *bnd;
  HM_CUDA_TRY(T.get((void **)&rows, sizeof(int32_t) * (size_t)(kW * m + kW)));
  HM_CUDA_TRY(T.get((void **)&tmp, sizeof(int32_t) * (size_t)(kW * m + kW)));
  HM_CUDA_TRY(T.get((void **)&out_off, sizeof(int64_t) * (size_t)(2 * (n + 1)) + 64));
  in_off = out_off + (n + 1);
  HM_CUDA_TRY(T.get((void **)&err, sizeof(uint32_t)));
  HM_CUDA_TRY(T.get((void **)&bnd, sizeof(Bounds)));
  HM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
  const Bounds init{INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN};
  HM_CUDA_TRY(cudaMemcpyAsync(bnd, &init, sizeof(Bounds), cudaMemcpyHostToDevice, s));

  if (m) k_pack<<<grid_for(m), kThreads, 0, s>>>(d_src, d_dst, d_elab, m, n, rows, err, bnd);
  if (n) k_vbounds<<<grid_for(n), kThreads, 0, s>>>(d_vlab, n, bnd);
  uint32_t h_err = 0;
  Bounds hb;
  HM_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  HM_CUDA_TRY(cudaMemcpyAsync(&hb, bnd, sizeof(Bounds), cudaMemcpyDeviceToHost, s));
  HM_CUDA_TRY(cudaStreamSynchronize(s));
  HM_CUDA_TRY(cudaGetLastError());
  if (h_err & kErrRange) return HM_ERR_ARG;
  if (h_err & kErrSelf) return HM_ERR_SELF_LOOP;

  HM_CUDA_TRY(dmalloc(&g->src, m));
  HM_CUDA_TRY(dmalloc(&g->out_adj, m));
  HM_CUDA_TRY(dmalloc(&g->out_elab, m));
  HM_CUDA_TRY(dmalloc(&g->in_adj, m));
  HM_CUDA_TRY(dmalloc(&g->in_elab, m));
  HM_CUDA_TRY(dmalloc(&g->vi, n));
  HM_CUDA_TRY(dmalloc(&g->off, n));
  HM_CUDA_TRY(dmalloc(&g->vdir, n));
  g->afilt_nblk = (uint32_t)std::max<int64_t>(1, (m + 7) / 8);
  HM_CUDA_TRY(dmalloc(&g->afilt, 2 * (int64_t)g->afilt_nblk));
  HM_CUDA_TRY(cudaMemsetAsync(g->afilt, 0, 32 * (size_t)g->afilt_nblk, s));
  g->ahash_nbkt = (uint32_t)std::max<int64_t>(1, m);
  HM_CUDA_TRY(dmalloc(&g->ahash, 2 * (int64_t)g->ahash_nbkt));
  HM_CUDA_TRY(cudaMemsetAsync(g->ahash, 0xff, 32 * (size_t)g->ahash_nbkt, s));

  const int nbits = bits_for(n);
  int be = 1, bv = 1;
  uint32_t xe = 0, xv = 0;
  if (m) label_key(hb.emin, hb.emax, &be, &xe);
  if (n) label_key(hb.vmin, hb.vmax, &bv, &xv);
  uint32_t *oidx = nullptr, *iidx = nullptr;
  if (m) {
    const int by_src[2] = {0, 1};
    const int by_dst[2] = {1, 0};
    hm_status st = radix_sort_rows(rows, tmp, m, kW, by_src, 2, nbits, s);
    if (st != HM_OK) return st;
    k_split<<<grid_for(m), kThreads, 0, s>>>(rows, m, n, 0, 1, g->src, g->out_adj, g->out_elab,
                                             out_off, err);
    k_filter<<<grid_for(m), kThreads, 0, s>>>(g->src, g->out_adj, g->out_elab, m, g->afilt_nblk,
                                              reinterpret_cast<uint32_t *>(g->afilt));
    k_hash<<<grid_for(m), kThreads, 0, s>>>(g->src, g->out_adj, g->out_elab, m, g->ahash_nbkt,
                                            g->ahash, err);
    st = build_groups(rows, tmp, m, n, 0, 1, d_vlab, out_off, nbits, be, xe, bv, xv, s, T,
                      &g->gout_adj, &g->gdir_out, &g->ndir_out, &oidx);
    if (st != HM_OK) return st;
    st = radix_sort_rows(rows, tmp, m, kW, by_dst, 2, nbits, s);
    if (st != HM_OK) return st;
    k_split<<<grid_for(m), kThreads, 0, s>>>(rows, m, n, 1, 0, nullptr, g->in_adj, g->in_elab,
                                             in_off, nullptr);
    st = build_groups(rows, tmp, m, n, 1, 0, d_vlab, in_off, nbits, be, xe, bv, xv, s, T,
                      &g->gin_adj, &g->gdir_in, &g->ndir_in, &iidx);
    if (st != HM_OK) return st;
  } else {
    k_zero_off<<<grid_for(n + 1), kThreads, 0, s>>>(out_off, n);
    k_zero_off<<<grid_for(n + 1), kThreads, 0, s>>>(in_off, n);
    HM_CUDA_TRY(dmalloc(&g->gout_adj, 1));
    HM_CUDA_TRY(dmalloc(&g->gin_adj, 1));
    HM_CUDA_TRY(dmalloc(&g->gdir_out, 1));
    HM_CUDA_TRY(dmalloc(&g->gdir_in, 1));
  }
  if (n)
    k_vertex<<<grid_for(n), kThreads, 0, s>>>(d_vlab, out_off, in_off, oidx, iidx, n, g->vi, g->off,
                                              g->vdir);
  HM_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  HM_CUDA_TRY(cudaStreamSynchronize(s));
  HM_CUDA_TRY(cudaGetLastError());
  if (h_err & kErrDup) return HM_ERR_DUP_EDGE;
  if (h_err & kErrHash) return HM_ERR_CUDA;  // cannot happen (twice as many slots as arcs)
  g->bytes = sizeof(int32_t) * 7 * (size_t)m + (sizeof(int4) * 2 + sizeof(int2)) * (size_t)n +
             sizeof(int4) * (size_t)(g->ndir_out + g->ndir_in) + 32 * (size_t)g->afilt_nblk +
             32 * (size_t)g->ahash_nbkt;
  return HM_OK;
}

void free_graph_arrays(hm_graph *g) {
  void *ptrs[] = {g->src,     g->out_adj,  g->out_elab, g->in_adj,   g->in_elab, g->vi,
                  g->off,     g->gout_adj, g->gin_adj,  g->gdir_out, g->gdir_in, g->vdir,
                  g->afilt,   g->ahash,    g->check};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

}  // namespace

extern "C" hm_status hm_load_graph(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                   const int32_t *vlab, const int32_t *elab, int device_ptrs,
                                   void *stream, hm_graph **out) {
  if (!out || n < 0 || m < 0 || m > INT64_C(0x7FFFFFFF)) return HM_ERR_ARG;
  if (m > 0 && (!src || !dst || !elab)) return HM_ERR_ARG;
  if (n > 0 && !vlab) return HM_ERR_ARG;
  if (m > 0 && n == 0) return HM_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    return HM_ERR_NO_DEVICE;
  }
  ensure_pool();
  cudaStream_t s = (cudaStream_t)stream;
  hm_graph *g = new hm_graph();
  std::memset(g, 0, sizeof(*g));
  cudaGetDevice(&g->device);
  g->n = n;
  g->m = m;
  hm_status st = load_graph_impl(n, m, src, dst, vlab, elab, device_ptrs, s, g);
  if (st == HM_OK && cudaStreamSynchronize(s) != cudaSuccess) st = HM_ERR_CUDA;
  if (st != HM_OK) {
    cudaStreamSynchronize(s);
    (void)cudaGetLastError();
    free_graph_arrays(g);
    delete g;
    return st;
  }
  *out = g;
  return HM_OK;
}

extern "C" void hm_free_graph(hm_graph *g) {
  if (!g) return;
  free_graph_arrays(g);
  free(g->vtab);
  free(g->etab);
  delete g;
}

extern "C" hm_status hm_check_status(const hm_graph *g, uint64_t *violation) {
  if (!g || !violation) return HM_ERR_ARG;
#if HM_CHECK
  unsigned long long w = 0;
  if (cudaMemcpy(&w, g->check, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(g->check, 0, sizeof(w)) != cudaSuccess)
    return HM_ERR_CUDA;
  *violation = w;
  return HM_OK;
#else
  *violation = 0;
  return HM_ERR_ARG;  // built without the bounds checks
#endif
}

extern "C" hm_status hm_graph_info(const hm_graph *g, int32_t *n, int64_t *m,
                                   size_t *device_bytes) {
  if (!g) return HM_ERR_ARG;
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (device_bytes) *device_bytes = g->bytes;
  return HM_OK;
}

extern "C" hm_status hm_graph_export(const hm_graph *g, int64_t *out_off, int32_t *out_adj,
                                     int32_t *out_elab, int64_t *in_off, int32_t *in_adj,
                                     int32_t *in_elab) {
  if (!g) return HM_ERR_ARG;
  const size_t m = (size_t)g->m, n = (size_t)g->n;
  if (out_adj && m) HM_CUDA_TRY(cudaMemcpy(out_adj, g->out_adj, 4 * m, cudaMemcpyDeviceToHost));
  if (out_elab && m) HM_CUDA_TRY(cudaMemcpy(out_elab, g->out_elab, 4 * m, cudaMemcpyDeviceToHost));
  if (in_adj && m) HM_CUDA_TRY(cudaMemcpy(in_adj, g->in_adj, 4 * m, cudaMemcpyDeviceToHost));
  if (in_elab && m) HM_CUDA_TRY(cudaMemcpy(in_elab, g->in_elab, 4 * m, cudaMemcpyDeviceToHost));
  if (out_off || in_off) {
    int2 *h = (int2 *)malloc(sizeof(int2) * (n ? n : 1));
    if (!h) return HM_ERR_OOM;
    cudaError_t e = n ? cudaMemcpy(h, g->off, sizeof(int2) * n, cudaMemcpyDeviceToHost)
                      : cudaSuccess;
    if (e != cudaSuccess) {
      free(h);
      return HM_ERR_CUDA;
    }
    for (size_t v = 0; v < n; ++v) {
      if (out_off) out_off[v] = h[v].x;
      if (in_off) in_off[v] = h[v].y;
    }
    if (out_off) out_off[n] = (int64_t)m;
    if (in_off) in_off[n] = (int64_t)m;
    free(h);
  }
  return HM_OK;
}

extern "C" hm_status hm_graph_export_groups(const hm_graph *g, int32_t *gout_adj,
                                            int32_t *gin_adj, int32_t *vdir, int32_t *gdir_out,
                                            int32_t *gdir_in, int64_t *ndir) {
  if (!g) return HM_ERR_ARG;
  const size_t m = (size_t)g->m, n = (size_t)g->n;
  if (ndir) {
    ndir[0] = g->ndir_out;
    ndir[1] = g->ndir_in;
  }
  if (gout_adj && m) HM_CUDA_TRY(cudaMemcpy(gout_adj, g->gout_adj, 4 * m, cudaMemcpyDeviceToHost));
  if (gin_adj && m) HM_CUDA_TRY(cudaMemcpy(gin_adj, g->gin_adj, 4 * m, cudaMemcpyDeviceToHost));
  if (vdir && n) HM_CUDA_TRY(cudaMemcpy(vdir, g->vdir, sizeof(int4) * n, cudaMemcpyDeviceToHost));
  if (gdir_out && g->ndir_out)
    HM_CUDA_TRY(cudaMemcpy(gdir_out, g->gdir_out, sizeof(int4) * g->ndir_out, cudaMemcpyDeviceToHost));
  if (gdir_in && g->ndir_in)
    HM_CUDA_TRY(cudaMemcpy(gdir_in, g->gdir_in, sizeof(int4) * g->ndir_in, cudaMemcpyDeviceToHost));
  return HM_OK;
}
