// hm_pattern.cpp -- pattern validation, Structural Reordering (Alg. 1) and the
// per-position plans the kernels run (host code; needs no GPU).
//
// Alg. 1 (Sec. III-A): rank sigma(v) = (totaldeg(v), outdeg(v)) compared
// lexicographically; the sigma-argmax goes to position 0; then, while vertices
// remain, the next position takes the sigma-argmax among the unplaced
// out-neighbours of the vertex placed last, or among all unplaced vertices if
// it has none.  Readings where the paper is silent or garbled:
//   * ties beyond outdeg go to the lowest original id;
//   * degrees are the pattern's static degrees (nothing is re-ranked);
//   * positions are 0-based (the listing's 1-based pi(1) is position 0);
//   * if the fallback pick has no arc to any placed vertex, the sigma-argmax
//     among unplaced vertices that do have one is taken instead, so every
//     position >= 1 has at least one arc to an earlier position (an anchor).
//
// Plan (what the kernels check at each position, Sec. III-B/C):
//   positions 0,1 -- the seeding arc: normally pattern arc 0->1, so a target
//     arc (a,b) proposes f(0)=a, f(1)=b; if the pattern only has 1->0, the
//     target arc (a,b) proposes f(1)=a, f(0)=b.  The edge validator's other
//     direction: required with its label when the pattern has both arcs,
//     forbidden in induced mode when the pattern has only one.
//   position p >= 2 -- for every earlier q: the pattern arcs between q and p
//     become "arc must exist with this label" conditions, and in induced mode
//     the missing ones become "arc must not exist" conditions.
#include <algorithm>
#include <array>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "hm_internal.cuh"

namespace {

struct PatternGraph {
  int k = 0;
  bool arc[HM_MAX_K][HM_MAX_K] = {};
  int32_t lab[HM_MAX_K][HM_MAX_K] = {};
  int32_t vlab[HM_MAX_K] = {};
  int indeg[HM_MAX_K] = {};
  int outdeg[HM_MAX_K] = {};
};

bool sigma_less(const PatternGraph &P, int a, int b) {
  int ta = P.indeg[a] + P.outdeg[a], tb = P.indeg[b] + P.outdeg[b];
  if (ta != tb) return ta < tb;
  return P.outdeg[a] < P.outdeg[b];
}

// sigma-argmax over the vertices flagged in `cand` (lowest id wins ties); -1 if none.
int argmax_sigma(const PatternGraph &P, const bool *cand) {
  int best = -1;
  for (int v = 0; v < P.k; ++v) {
    if (!cand[v]) continue;
    if (best < 0 || sigma_less(P, best, v)) best = v;
  }
  return best;
}

void structural_reorder(const PatternGraph &P, int32_t *order) {
  bool placed[HM_MAX_K] = {};
  bool cand[HM_MAX_K];
  for (int v = 0; v < P.k; ++v) cand[v] = true;
  int n_placed = 0;
  order[n_placed] = argmax_sigma(P, cand);
  placed[order[n_placed++]] = true;
  while (n_placed < P.k) {
    int u = order[n_placed - 1];
    bool any = false;
    for (int w = 0; w < P.k; ++w) {
      cand[w] = !placed[w] && P.arc[u][w];
      any |= cand[w];
    }
    int w_star;
    if (any) {
      w_star = argmax_sigma(P, cand);
    } else {
      for (int w = 0; w < P.k; ++w) cand[w] = !placed[w];
      w_star = argmax_sigma(P, cand);
      bool anchored = false;
      for (int r = 0; r < P.k; ++r)
        if (placed[r] && (P.arc[w_star][r] || P.arc[r][w_star])) anchored = true;
      if (!anchored) {
        bool found = false;
        for (int w = 0; w < P.k; ++w) {
          cand[w] = false;
          if (placed[w]) continue;
          for (int r = 0; r < P.k; ++r)
            if (placed[r] && (P.arc[w][r] || P.arc[r][w])) cand[w] = true;
          found |= cand[w];
        }
        if (found) w_star = argmax_sigma(P, cand);
      }
    }
    order[n_placed++] = w_star;
    placed[w_star] = true;
  }
}

void build_plan(const PatternGraph &P, const int32_t *order, int induced, hm::Plan &pl) {
  std::memset(&pl, 0, sizeof(pl));
  const int k = P.k;
  pl.k = k;
  pl.induced = induced;
  pl.root_pos = -1;
  bool A[HM_MAX_K][HM_MAX_K];
  int32_t L[HM_MAX_K][HM_MAX_K];
  for (int i = 0; i < k; ++i) {
    pl.orig[i] = order[i];
    pl.vlab[i] = P.vlab[order[i]];
    pl.din[i] = P.indeg[order[i]];
    pl.dout[i] = P.outdeg[order[i]];
    for (int j = 0; j < k; ++j) {
      A[i][j] = P.arc[order[i]][order[j]];
      L[i][j] = P.lab[order[i]][order[j]];
    }
  }
  if (A[0][1]) {
    pl.seed_rev = 0;
    pl.seed_lab = L[0][1];
    pl.back_req = A[1][0] ? 1 : 0;
    pl.back_lab = A[1][0] ? L[1][0] : 0;
    pl.back_forbid = (induced && !A[1][0]) ? 1 : 0;
  } else {
    pl.seed_rev = 1;
    pl.seed_lab = L[1][0];
    pl.back_req = 0;
    pl.back_lab = 0;
    pl.back_forbid = induced ? 1 : 0;
  }
  int ov = 0;
  for (int w = 2; w < k; ++w)
    if ((A[0][w] || A[w][0]) && (A[1][w] || A[w][1])) ++ov;
  pl.ov_need = ov;
  // position 1 has no pattern arc to any later position: its image can be chosen last
  pl.defer1 = k >= 3;
  for (int p = 2; p < k; ++p)
    if (A[1][p] || A[p][1]) pl.defer1 = 0;
  int slots = 0;
  for (int p = 2; p < k; ++p) {
    int c = 0;
    pl.gbase[p] = slots;
    for (int q = 0; q < p; ++q) {
      if (A[q][p]) pl.cons[p][c++] = hm::Cons{(int8_t)q, hm::kOut, 0, L[q][p]};
      if (A[p][q]) pl.cons[p][c++] = hm::Cons{(int8_t)q, hm::kIn, 0, L[p][q]};
    }
    pl.npos[p] = c;
    slots += c;
    if (induced) {
      for (int q = 0; q < p; ++q) {
        if (!A[q][p]) pl.cons[p][c++] = hm::Cons{(int8_t)q, hm::kNotOut, 0, 0};
        if (!A[p][q]) pl.cons[p][c++] = hm::Cons{(int8_t)q, hm::kNotIn, 0, 0};
      }
    }
    pl.ncons[p] = c;
  }
  pl.ngrp = slots;
  // look-ahead classes: the pattern arcs from each position to later ones
  for (int p = 0; p < k; ++p) {
    int n = 0;
    for (int w = p + 1; w < k; ++w)
      for (int dir = 0; dir < 2; ++dir) {
        const bool arc = dir == 0 ? A[p][w] : A[w][p];
        if (!arc) continue;
        const int32_t alab = dir == 0 ? L[p][w] : L[w][p];
        const int32_t vl = P.vlab[order[w]];
        int c = 0;
        while (c < n && !(pl.la[p][c].kind == (dir == 0 ? hm::kOut : hm::kIn) && pl.la[p][c].alab == alab &&
                          pl.la[p][c].vlab == vl))
          ++c;
        if (c == n) pl.la[p][n++] = hm::LookClass{(int8_t)(dir == 0 ? hm::kOut : hm::kIn), 0, 0, alab, vl};
        pl.la[p][c].need++;
      }
    pl.nla[p] = n;
  }
}

// ---- symmetry breaking ---------------------------------------------------------
//
// An automorphism of the labelled pattern is a permutation s of its vertices
// that keeps every vertex label and maps every arc onto an arc with the same
// label (so non-arcs onto non-arcs).  If f is a match (Eqs. 1-3, either mode),
// so is f o s, and the |Aut| maps f o s are distinct: the matches fall into
// orbits of exactly |Aut|.  Order constraints chosen as by Grochow and Kellis
// (RECOMB 2007) keep exactly one map per orbit: while the group G is not
// trivial, take a vertex v of a largest G-orbit, require f(v) < f(w) for every
// other w in that orbit, and continue with the stabiliser of v.  (For any f
// the images f o s, s in G, that satisfy the first constraints are those
// sending v to the orbit member with the smallest image: a coset of the
// stabiliser, on which the next constraints act the same way.)

using Perm = std::array<int8_t, HM_MAX_K>;

// Every automorphism by backtracking over the vertices in id order; false
// when there are more than `cap`.
bool enumerate_automorphisms(const PatternGraph &P, int cap, std::vector<Perm> &out) {
  const int k = P.k;
  Perm s{};
  bool used[HM_MAX_K] = {};
  bool over = false;
  auto rec = [&](auto &&self, int i) -> void {
    if (over) return;
    if (i == k) {
      if ((int)out.size() >= cap) {
        over = true;
        return;
      }
      out.push_back(s);
      return;
    }
    for (int u = 0; u < k && !over; ++u) {
      if (used[u] || P.vlab[u] != P.vlab[i] || P.indeg[u] != P.indeg[i] || P.outdeg[u] != P.outdeg[i])
        continue;
      bool ok = true;
      for (int j = 0; j < i && ok; ++j) {
        const int sj = s[j];
        if (P.arc[i][j] != P.arc[u][sj] || (P.arc[i][j] && P.lab[i][j] != P.lab[u][sj])) ok = false;
        if (P.arc[j][i] != P.arc[sj][u] || (P.arc[j][i] && P.lab[j][i] != P.lab[sj][u])) ok = false;
      }
      if (!ok) continue;
      s[i] = (int8_t)u;
      used[u] = true;
      self(self, i + 1);
      used[u] = false;
    }
  };
  rec(rec, 0);
  return !over;
}

// Fills the plans' symmetry fields for the search order `order` (position ->
// original vertex); leaves naut = 1 (no symmetry breaking) for two-vertex
// patterns and for patterns with more than kMaxAut automorphisms.
void add_symmetry(const PatternGraph &P, const int32_t *order, hm::Plan *plans, int nplans) {
  const int k = P.k;
  int pos[HM_MAX_K];
  for (int i = 0; i < k; ++i) pos[order[i]] = i;
  for (int m = 0; m < nplans; ++m) {
    hm::Plan &pl = plans[m];
    pl.naut = 1;
    for (int v = 0; v < k; ++v) pl.aut[0][v] = (int8_t)pos[v];
    for (int p = 0; p < k; ++p) pl.sym_gt[p] = pl.sym_lt[p] = 0;
  }
  if (k < 3) return;
  std::vector<Perm> group;
  if (!enumerate_automorphisms(P, hm::kMaxAut, group) || group.size() <= 1) return;
  // constraints f(v) < f(w), as pairs of original vertices
  std::vector<std::pair<int, int>> lt;
  std::vector<Perm> G = group;
  while (G.size() > 1) {
    int best = -1, best_size = 0;
    bool in_orbit[HM_MAX_K][HM_MAX_K] = {};
    int orbit_size[HM_MAX_K] = {};
    for (int v = 0; v < k; ++v) {
      for (const Perm &g : G) in_orbit[v][g[v]] = true;
      for (int w = 0; w < k; ++w) orbit_size[v] += in_orbit[v][w];
    }
    for (int v = 0; v < k; ++v)  // a largest orbit; among its vertices, the earliest in the search order
      if (orbit_size[v] > best_size || (orbit_size[v] == best_size && best >= 0 && pos[v] < pos[best])) {
        best = v;
        best_size = orbit_size[v];
      }
    for (int w = 0; w < k; ++w)
      if (w != best && in_orbit[best][w]) lt.emplace_back(best, w);
    std::vector<Perm> stab;
    for (const Perm &g : G)
      if (g[best] == best) stab.push_back(g);
    G.swap(stab);
  }
  for (int m = 0; m < nplans; ++m) {
    hm::Plan &pl = plans[m];
    pl.naut = (int32_t)group.size();
    for (size_t si = 0; si < group.size(); ++si)
      for (int v = 0; v < k; ++v) pl.aut[si][v] = (int8_t)pos[group[si][v]];
    for (const auto &c : lt) {
      const int pv = pos[c.first], pw = pos[c.second];  // f(v) < f(w)
      if (pv < pw) pl.sym_gt[pw] |= 1u << pv;  // checked when w is mapped: f(w) > f(v)
      else pl.sym_lt[pv] |= 1u << pw;          // checked when v is mapped: f(v) < f(w)
    }
  }
}

bool weakly_connected(const PatternGraph &P) {
  int parent[HM_MAX_K];
  for (int i = 0; i < P.k; ++i) parent[i] = i;
  auto find = [&](int x) {
    while (parent[x] != x) x = parent[x] = parent[parent[x]];
    return x;
  };
  for (int a = 0; a < P.k; ++a)
    for (int b = 0; b < P.k; ++b)
      if (P.arc[a][b]) parent[find(a)] = find(b);
  int root = find(0);
  for (int i = 1; i < P.k; ++i)
    if (find(i) != root) return false;
  return true;
}

}  // namespace

extern "C" hm_status hm_load_pattern(int32_t k, int32_t mp, const int32_t *src,
                                     const int32_t *dst, const int32_t *vlab,
                                     const int32_t *elab, hm_pattern **out) {
  if (!out || !vlab || mp < 0) return HM_ERR_ARG;
  if (k < 2 || k > HM_MAX_K || mp < 1) return HM_ERR_PATTERN;
  if (!src || !dst || !elab) return HM_ERR_ARG;
  PatternGraph P;
  P.k = k;
  for (int i = 0; i < k; ++i) P.vlab[i] = vlab[i];
  for (int e = 0; e < mp; ++e) {
    int a = src[e], b = dst[e];
    if (a < 0 || a >= k || b < 0 || b >= k) return HM_ERR_ARG;
    if (a == b) return HM_ERR_SELF_LOOP;
    if (P.arc[a][b]) return HM_ERR_DUP_EDGE;
    P.arc[a][b] = true;
    P.lab[a][b] = elab[e];
    P.outdeg[a]++;
    P.indeg[b]++;
  }
  if (!weakly_connected(P)) return HM_ERR_PATTERN;
  hm_pattern *p = new (std::nothrow) hm_pattern();
  if (!p) return HM_ERR_OOM;
  p->k = k;
  p->mp = mp;
  structural_reorder(P, p->order);
  build_plan(P, p->order, 0, p->plan[0]);
  build_plan(P, p->order, 1, p->plan[1]);
  add_symmetry(P, p->order, p->plan, 2);
  *out = p;
  return HM_OK;
}

extern "C" hm_status hm_load_pattern_ordered(int32_t k, int32_t mp, const int32_t *src,
                                             const int32_t *dst, const int32_t *vlab,
                                             const int32_t *elab, const int32_t *order,
                                             hm_pattern **out) {
  if (!order) return HM_ERR_ARG;
  hm_pattern *p = nullptr;
  hm_status st = hm_load_pattern(k, mp, src, dst, vlab, elab, &p);  // validation + Alg. 1
  if (st != HM_OK) return st;
  PatternGraph P;
  P.k = k;
  for (int i = 0; i < k; ++i) P.vlab[i] = vlab[i];
  for (int e = 0; e < mp; ++e) {
    P.arc[src[e]][dst[e]] = true;
    P.lab[src[e]][dst[e]] = elab[e];
    P.outdeg[src[e]]++;
    P.indeg[dst[e]]++;
  }
  // the given order must be a permutation in which every position after the
  // first has an arc (either direction) to an earlier position
  bool seen[HM_MAX_K] = {};
  for (int i = 0; i < k; ++i) {
    const int v = order[i];
    if (v < 0 || v >= k || seen[v]) {
      hm_free_pattern(p);
      return HM_ERR_ARG;
    }
    bool anchored = i == 0;
    for (int j = 0; j < i; ++j)
      if (P.arc[v][order[j]] || P.arc[order[j]][v]) anchored = true;
    if (!anchored) {
      hm_free_pattern(p);
      return HM_ERR_PATTERN;
    }
    seen[v] = true;
  }
  for (int i = 0; i < k; ++i) p->order[i] = order[i];
  build_plan(P, p->order, 0, p->plan[0]);
  build_plan(P, p->order, 1, p->plan[1]);
  add_symmetry(P, p->order, p->plan, 2);
  *out = p;
  return HM_OK;
}

extern "C" void hm_free_pattern(hm_pattern *p) { delete p; }

extern "C" hm_status hm_pattern_automorphisms(const hm_pattern *p, int32_t *count) {
  if (!p || !count) return HM_ERR_ARG;
  *count = p->plan[0].naut;
  return HM_OK;
}

extern "C" hm_status hm_pattern_order(const hm_pattern *p, int32_t *order_out) {
  if (!p || !order_out) return HM_ERR_ARG;
  for (int i = 0; i < p->k; ++i) order_out[i] = p->order[i];
  return HM_OK;
}
