// hm_props.cpp -- several properties per vertex and per arc (host code).
//
// checkAttributes of the vertex and edge validators (Alg. 2, Alg. 3) compares
// every property of a vertex or an arc (Sec. III-D supports arbitrary numbers
// of properties).  Two property tuples are equal exactly when their ranks in
// the sorted list of distinct tuples are equal, so the graph is loaded with
// each tuple replaced by that rank and every kernel compares one int32 as
// before.  The sorted tuple tables stay with the graph; a pattern's tuples are
// looked up in them, and a tuple the graph does not have becomes -1, a label
// no target vertex or arc carries.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "hm_internal.cuh"

namespace {

bool tuple_less(const int32_t *a, const int32_t *b, int32_t w) {
  for (int32_t i = 0; i < w; ++i)
    if (a[i] != b[i]) return a[i] < b[i];
  return false;
}

// ids[i] = rank of row i among the distinct rows; table = the distinct rows, sorted.
void rank_tuples(int64_t count, int32_t w, const int32_t *rows, std::vector<int32_t> &ids,
                 std::vector<int32_t> &table) {
  std::vector<int64_t> order((size_t)count);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
    return tuple_less(rows + x * w, rows + y * w, w);
  });
  ids.assign((size_t)count, 0);
  table.clear();
  int32_t rank = -1;
  for (int64_t i = 0; i < count; ++i) {
    const int32_t *r = rows + order[i] * w;
    if (i == 0 || tuple_less(rows + order[i - 1] * w, r, w)) {
      ++rank;
      table.insert(table.end(), r, r + w);
    }
    ids[(size_t)order[i]] = rank;
  }
}

int32_t lookup_tuple(const int32_t *table, int64_t ntab, int32_t w, const int32_t *t) {
  int64_t lo = 0, hi = ntab;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (tuple_less(table + mid * w, t, w)) lo = mid + 1; else hi = mid;
  }
  return (lo < ntab && !tuple_less(t, table + lo * w, w)) ? (int32_t)lo : -1;
}

}  // namespace

extern "C" hm_status hm_load_graph_props(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                         int32_t nvp, const int32_t *vprops, int32_t nep,
                                         const int32_t *eprops, void *stream, hm_graph **out) {
  if (!out || n < 0 || m < 0 || nvp < 1 || nep < 1 || nvp > 64 || nep > 64) return HM_ERR_ARG;
  if ((n > 0 && !vprops) || (m > 0 && (!eprops || !src || !dst))) return HM_ERR_ARG;
  std::vector<int32_t> vids, eids, vtab, etab;
  rank_tuples(n, nvp, vprops, vids, vtab);
  rank_tuples(m, nep, eprops, eids, etab);
  hm_graph *g = nullptr;
  const hm_status st = hm_load_graph(n, m, src, dst, vids.data(), eids.data(), 0, stream, &g);
  if (st != HM_OK) return st;
  g->nvp = nvp;
  g->nep = nep;
  g->nvtab = (int64_t)(vtab.size() / (size_t)nvp);
  g->netab = (int64_t)(etab.size() / (size_t)nep);
  g->vtab = (int32_t *)malloc(sizeof(int32_t) * std::max<size_t>(vtab.size(), 1));
  g->etab = (int32_t *)malloc(sizeof(int32_t) * std::max<size_t>(etab.size(), 1));
  if (!g->vtab || !g->etab) {
    hm_free_graph(g);
    return HM_ERR_OOM;
  }
  if (!vtab.empty()) std::memcpy(g->vtab, vtab.data(), sizeof(int32_t) * vtab.size());
  if (!etab.empty()) std::memcpy(g->etab, etab.data(), sizeof(int32_t) * etab.size());
  *out = g;
  return HM_OK;
}

extern "C" hm_status hm_load_pattern_props(const hm_graph *g, int32_t k, int32_t mp,
                                           const int32_t *src, const int32_t *dst,
                                           const int32_t *vprops, const int32_t *eprops,
                                           hm_pattern **out) {
  if (!g || !out || !g->vtab || !g->etab) return HM_ERR_ARG;
  if (k < 2 || k > HM_MAX_K || mp < 1) return HM_ERR_PATTERN;
  if (!vprops || !eprops) return HM_ERR_ARG;
  std::vector<int32_t> vl((size_t)k), el((size_t)mp);
  for (int32_t i = 0; i < k; ++i) vl[i] = lookup_tuple(g->vtab, g->nvtab, g->nvp, vprops + (int64_t)i * g->nvp);
  for (int32_t e = 0; e < mp; ++e) el[e] = lookup_tuple(g->etab, g->netab, g->nep, eprops + (int64_t)e * g->nep);
  return hm_load_pattern(k, mp, src, dst, vl.data(), el.data(), out);
}
