/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this file's library.  The product path never calls it, and it shares
 * no code, header, table or helper with the CUDA library.
 *
 * What it computes (Sec. II-A, Eqs. 1-3).  Given a pattern G1 = (V1, E1) and a
 * target G2 = (V2, E2), both directed, with vertex labels alpha_i and edge
 * labels beta_i, it enumerates every injective f : V1 -> V2 such that
 *   Eq. (2)  alpha_1(v) = alpha_2(f(v))               for all v in V1,
 *   Eq. (3)  (f(u), f(v)) in E2 and beta_1(u, v) = beta_2(f(u), f(v))
 *                                                    for all (u, v) in E1,
 *   Eq. (1)  (u, v) in E1  <=>  (f(u), f(v)) in E2   (induced mode), or only
 *            "=>" (monomorphism, the relaxation stated right after Eq. 3).
 * A match is one such map (the method returns a list of mappings), so
 * automorphic copies count separately.  Rows are written as
 * (f(0), f(1), ..., f(k-1)) in the pattern's ORIGINAL vertex numbering and
 * returned sorted ascending lexicographically.
 *
 * How: plain backtracking from the EMPTY mapping.  Pattern vertices are
 * visited in breadth-first order over the undirected pattern, starting at
 * original vertex 0, neighbours in ascending order (a component that BFS
 * does not reach starts again at its lowest vertex).  A vertex with an
 * already-mapped BFS parent q takes its candidates from the target
 * out-list (pattern arc q->p) or in-list (arc p->q) of f(q); a BFS root
 * takes every target vertex.  Each candidate is accepted only if it is
 * unused, has the right label, and every pair with every mapped vertex
 * satisfies Eqs. (1) and (3) in both directions.  There is no reordering,
 * no vertex or edge validator and no degree filter: the visiting order
 * cannot change the set of maps that satisfy the definition.
 *
 * Target storage: out- and in-lists sorted by neighbour id, each entry
 * carrying its arc label; an arc lookup is a binary search in the
 * out-list.  The target must be simple (no self-loop, no repeated (u, v));
 * og_graph_new rejects anything else.
 *
 * Parallelism: POSIX threads take chunks of the first visited vertex's
 * candidates from a shared counter; each thread keeps its own count and row
 * buffer, merged and sorted at the end.
 *
 * Parity status: pinned (see the tests: brute force over all injective maps,
 * closed forms on complete digraphs, the labelled 3-cycle trace identity,
 * the automorphism identity and the monomorphism/induced completion sum).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_MAXK 24

enum { OG_OK = 0, OG_EARG = -1, OG_ESELF = -2, OG_EDUP = -3, OG_ENOMEM = -4 };

typedef struct og_graph {
  int32_t n;
  int64_t m;
  int64_t *out_start; /* n+1 */
  int32_t *out_nbr;   /* m, ascending within each vertex */
  int32_t *out_lab;
  int64_t *in_start;
  int32_t *in_nbr;
  int32_t *in_lab;
  int32_t *vlab; /* n */
} og_graph;

typedef struct {
  int32_t nbr, lab;
} og_pair;

static int cmp_pair(const void *a, const void *b) {
  const og_pair *x = (const og_pair *)a, *y = (const og_pair *)b;
  return (x->nbr > y->nbr) - (x->nbr < y->nbr);
}

/* Bucket the arcs by `key`, then sort each bucket by neighbour id. */
static int build_lists(int32_t n, int64_t m, const int32_t *key, const int32_t *other,
                       const int32_t *lab, int64_t **start_out, int32_t **nbr_out,
                       int32_t **lab_out) {
  int64_t *start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  og_pair *tmp = (og_pair *)malloc((size_t)(m > 0 ? m : 1) * sizeof(og_pair));
  int32_t *nbr = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int32_t *lb = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  if (!start || !fill || !tmp || !nbr || !lb) {
    free(start); free(fill); free(tmp); free(nbr); free(lb);
    return OG_ENOMEM;
  }
  for (int64_t e = 0; e < m; ++e) start[key[e] + 1]++;
  for (int32_t v = 0; v < n; ++v) start[v + 1] += start[v];
  memcpy(fill, start, ((size_t)n + 1) * sizeof(int64_t));
  for (int64_t e = 0; e < m; ++e) {
    int64_t at = fill[key[e]]++;
    tmp[at].nbr = other[e];
    tmp[at].lab = lab[e];
  }
  for (int32_t v = 0; v < n; ++v) {
    int64_t len = start[v + 1] - start[v];
    if (len > 1) qsort(tmp + start[v], (size_t)len, sizeof(og_pair), cmp_pair);
  }
  for (int64_t e = 0; e < m; ++e) {
    nbr[e] = tmp[e].nbr;
    lb[e] = tmp[e].lab;
  }
  free(fill);
  free(tmp);
  *start_out = start;
  *nbr_out = nbr;
  *lab_out = lb;
  return OG_OK;
}

void og_graph_free(og_graph *g) {
  if (!g) return;
  free(g->out_start); free(g->out_nbr); free(g->out_lab);
  free(g->in_start); free(g->in_nbr); free(g->in_lab);
  free(g->vlab);
  free(g);
}

int og_graph_new(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                 const int32_t *vlab, const int32_t *elab, og_graph **out) {
  if (n < 0 || m < 0 || !out || (m > 0 && (!src || !dst || !elab)) || (n > 0 && !vlab))
    return OG_EARG;
  for (int64_t e = 0; e < m; ++e) {
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return OG_EARG;
    if (src[e] == dst[e]) return OG_ESELF;
  }
  og_graph *g = (og_graph *)calloc(1, sizeof(og_graph));
  if (!g) return OG_ENOMEM;
  g->n = n;
  g->m = m;
  g->vlab = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!g->vlab) { og_graph_free(g); return OG_ENOMEM; }
  if (n > 0) memcpy(g->vlab, vlab, (size_t)n * sizeof(int32_t));
  if (build_lists(n, m, src, dst, elab, &g->out_start, &g->out_nbr, &g->out_lab) ||
      build_lists(n, m, dst, src, elab, &g->in_start, &g->in_nbr, &g->in_lab)) {
    og_graph_free(g);
    return OG_ENOMEM;
  }
  for (int32_t v = 0; v < n; ++v)
    for (int64_t i = g->out_start[v] + 1; i < g->out_start[v + 1]; ++i)
      if (g->out_nbr[i] == g->out_nbr[i - 1]) { og_graph_free(g); return OG_EDUP; }
  *out = g;
  return OG_OK;
}

/* Is (a, b) an arc of the target?  If so, store its label in *lab. */
static int target_arc(const og_graph *g, int32_t a, int32_t b, int32_t *lab) {
  int64_t lo = g->out_start[a], hi = g->out_start[a + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    int32_t x = g->out_nbr[mid];
    if (x == b) { *lab = g->out_lab[mid]; return 1; }
    if (x < b) lo = mid + 1; else hi = mid;
  }
  return 0;
}

typedef struct {
  int k;
  int arc[OG_MAXK][OG_MAXK];     /* arc[a][b] = 1 iff (a, b) in E1 */
  int32_t alab[OG_MAXK][OG_MAXK];/* beta_1(a, b) where arc[a][b] */
  int32_t vlab[OG_MAXK];
  int order[OG_MAXK];            /* visiting order, original ids */
  int parent[OG_MAXK];           /* BFS parent (original id) or -1 for a root */
  int from_parent[OG_MAXK];      /* 1: candidates from out(f(parent)); 0: from in(...) */
} og_pattern;

typedef struct {
  int32_t *data;
  size_t len, cap; /* in rows */
} og_rows;

typedef struct {
  const og_graph *g;
  const og_pattern *P;
  int induced;
  int want_rows;
  const uint8_t *root_mask;
  int64_t *next_root;   /* shared chunk counter */
  int failed;
  int32_t f[OG_MAXK];   /* f[original pattern vertex] */
  uint64_t count;
  og_rows rows;
} og_worker;

static int emit(og_worker *w) {
  w->count++;
  if (!w->want_rows) return 0;
  int k = w->P->k;
  if (w->rows.len == w->rows.cap) {
    size_t nc = w->rows.cap ? 2 * w->rows.cap : 1024;
    int32_t *nd = (int32_t *)realloc(w->rows.data, nc * (size_t)k * sizeof(int32_t));
    if (!nd) return -1;
    w->rows.data = nd;
    w->rows.cap = nc;
  }
  memcpy(w->rows.data + w->rows.len * (size_t)k, w->f, (size_t)k * sizeof(int32_t));
  w->rows.len++;
  return 0;
}

/* Can the pattern vertex p (visited at depth d) take target vertex c? */
static int feasible(const og_worker *w, int d, int p, int32_t c) {
  const og_graph *g = w->g;
  const og_pattern *P = w->P;
  if (g->vlab[c] != P->vlab[p]) return 0;                 /* Eq. (2) */
  for (int i = 0; i < d; ++i)
    if (w->f[P->order[i]] == c) return 0;                 /* injective */
  for (int i = 0; i < d; ++i) {
    int q = P->order[i];
    int32_t lab;
    /* the pair (q, p) */
    int present = target_arc(g, w->f[q], c, &lab);
    if (P->arc[q][p]) {
      if (!present || lab != P->alab[q][p]) return 0;     /* Eq. (3) */
    } else if (w->induced && present) {
      return 0;                                           /* Eq. (1), "<=" */
    }
    /* the pair (p, q) */
    present = target_arc(g, c, w->f[q], &lab);
    if (P->arc[p][q]) {
      if (!present || lab != P->alab[p][q]) return 0;
    } else if (w->induced && present) {
      return 0;
    }
  }
  return 1;
}

static int extend(og_worker *w, int d) {
  const og_pattern *P = w->P;
  const og_graph *g = w->g;
  if (d == P->k) return emit(w);
  int p = P->order[d];
  int q = P->parent[p];
  if (q < 0) {
    for (int32_t c = 0; c < g->n; ++c) {
      if (!feasible(w, d, p, c)) continue;
      w->f[p] = c;
      if (extend(w, d + 1)) return -1;
    }
    return 0;
  }
  int32_t fq = w->f[q];
  const int32_t *nbr;
  int64_t lo, hi;
  if (P->from_parent[p]) {
    nbr = g->out_nbr; lo = g->out_start[fq]; hi = g->out_start[fq + 1];
  } else {
    nbr = g->in_nbr; lo = g->in_start[fq]; hi = g->in_start[fq + 1];
  }
  for (int64_t i = lo; i < hi; ++i) {
    int32_t c = nbr[i];
    if (!feasible(w, d, p, c)) continue;
    w->f[p] = c;
    if (extend(w, d + 1)) return -1;
  }
  return 0;
}

static void *worker_main(void *arg) {
  og_worker *w = (og_worker *)arg;
  const int64_t chunk = 64;
  int p0 = w->P->order[0];
  for (;;) {
    int64_t begin = __atomic_fetch_add(w->next_root, chunk, __ATOMIC_RELAXED);
    if (begin >= w->g->n) break;
    int64_t end = begin + chunk < w->g->n ? begin + chunk : w->g->n;
    for (int64_t c = begin; c < end; ++c) {
      if (w->root_mask && !w->root_mask[c]) continue;
      if (!feasible(w, 0, p0, (int32_t)c)) continue;
      w->f[p0] = (int32_t)c;
      if (extend(w, 1)) { w->failed = 1; return NULL; }
    }
  }
  return NULL;
}

static int g_row_k; /* row width for the comparator (set before each sort) */
static pthread_mutex_t g_sort_lock = PTHREAD_MUTEX_INITIALIZER;

static int cmp_row(const void *a, const void *b) {
  const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
  for (int i = 0; i < g_row_k; ++i)
    if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}

static int make_pattern(int32_t k, int32_t mp, const int32_t *psrc, const int32_t *pdst,
                        const int32_t *pvlab, const int32_t *pelab, og_pattern *P) {
  if (k < 1 || k > OG_MAXK || mp < 0 || !pvlab || (mp > 0 && (!psrc || !pdst || !pelab)))
    return OG_EARG;
  memset(P, 0, sizeof(*P));
  P->k = k;
  for (int i = 0; i < k; ++i) P->vlab[i] = pvlab[i];
  for (int e = 0; e < mp; ++e) {
    int a = psrc[e], b = pdst[e];
    if (a < 0 || a >= k || b < 0 || b >= k) return OG_EARG;
    if (a == b) return OG_ESELF;
    if (P->arc[a][b]) return OG_EDUP;
    P->arc[a][b] = 1;
    P->alab[a][b] = pelab[e];
  }
  /* breadth-first visiting order over the undirected pattern */
  int seen[OG_MAXK] = {0};
  int nvis = 0;
  for (int root = 0; root < k; ++root) {
    if (seen[root]) continue;
    seen[root] = 1;
    P->parent[root] = -1;
    P->order[nvis++] = root;
    for (int head = nvis - 1; head < nvis; ++head) {
      int x = P->order[head];
      for (int y = 0; y < k; ++y) {
        if (seen[y] || !(P->arc[x][y] || P->arc[y][x])) continue;
        seen[y] = 1;
        P->parent[y] = x;
        P->from_parent[y] = P->arc[x][y] ? 1 : 0;
        P->order[nvis++] = y;
      }
    }
  }
  return OG_OK;
}

/*
 * Enumerate the matches of the pattern in `g`.
 *   mode: 0 = monomorphism, 1 = induced subgraph isomorphism.
 *   root_mask: NULL, or uint8[n]; when given, only maps with
 *              root_mask[f(0)] != 0 are counted (original vertex 0).
 *   want_rows: when non-zero, *rows receives count*k int32 (malloc'ed,
 *              free with og_rows_free), sorted lexicographically.
 */
int og_match(const og_graph *g, int32_t k, int32_t mp, const int32_t *psrc,
             const int32_t *pdst, const int32_t *pvlab, const int32_t *pelab, int mode,
             int nthreads, const uint8_t *root_mask, int want_rows, uint64_t *count,
             int32_t **rows) {
  if (!g || !count || (mode != 0 && mode != 1) || (want_rows && !rows)) return OG_EARG;
  og_pattern P;
  int rc = make_pattern(k, mp, psrc, pdst, pvlab, pelab, &P);
  if (rc) return rc;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  int64_t next_root = 0;
  og_worker *ws = (og_worker *)calloc((size_t)nthreads, sizeof(og_worker));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!ws || !th) { free(ws); free(th); return OG_ENOMEM; }
  for (int t = 0; t < nthreads; ++t) {
    ws[t].g = g;
    ws[t].P = &P;
    ws[t].induced = mode;
    ws[t].want_rows = want_rows;
    ws[t].root_mask = root_mask;
    ws[t].next_root = &next_root;
  }
  int started = 0;
  for (int t = 1; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, worker_main, &ws[t]) != 0) break;
    started = t;
  }
  worker_main(&ws[0]);
  for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
  uint64_t total = 0;
  size_t nrows = 0;
  int failed = 0;
  for (int t = 0; t < nthreads; ++t) {
    total += ws[t].count;
    nrows += ws[t].rows.len;
    failed |= ws[t].failed;
  }
  int32_t *all = NULL;
  if (!failed && want_rows) {
    all = (int32_t *)malloc((nrows ? nrows : 1) * (size_t)k * sizeof(int32_t));
    if (!all) failed = 1;
    size_t at = 0;
    for (int t = 0; all && t < nthreads; ++t) {
      memcpy(all + at * (size_t)k, ws[t].rows.data, ws[t].rows.len * (size_t)k * sizeof(int32_t));
      at += ws[t].rows.len;
    }
    if (all && nrows > 1) {
      pthread_mutex_lock(&g_sort_lock);
      g_row_k = k;
      qsort(all, nrows, (size_t)k * sizeof(int32_t), cmp_row);
      pthread_mutex_unlock(&g_sort_lock);
    }
  }
  for (int t = 0; t < nthreads; ++t) free(ws[t].rows.data);
  free(ws);
  free(th);
  if (failed) { free(all); return OG_ENOMEM; }
  *count = total;
  if (want_rows) *rows = all;
  return OG_OK;
}

void og_rows_free(int32_t *rows) { free(rows); }

/* Copy out the sorted out-list of v (for tests of the loader's sort order). */
int64_t og_out_degree(const og_graph *g, int32_t v) {
  if (!g || v < 0 || v >= g->n) return -1;
  return g->out_start[v + 1] - g->out_start[v];
}
