"""The method's own host-side steps, written out plainly -- TEST INFRASTRUCTURE ONLY.

These follow the paper's algorithms step by step, in its order and notation,
so the CUDA path's intermediate results can be checked against them:

  * :func:`structural_reorder` -- Alg. 1 (Structural Reordering, Sec. III-A):
    rank sigma(v) = (totaldeg(v), outdeg(v)); place the sigma-argmax first;
    then repeatedly take the sigma-argmax among the unplaced out-neighbours of
    the last placed vertex, or among all unplaced vertices when there are none.
  * :func:`vertex_flags` -- Alg. 2 (Vertex Validator, Sec. III-B).
  * :func:`edge_validator` / :func:`injected_states` -- Alg. 3 (Edge
    Validator) applied inside the edge loop of the HiPerMotif algorithm
    (Sec. III-C): every target arc is tried as the image of the reordered
    pattern arc between positions 0 and 1; survivors become depth-2 states.

Readings taken where the paper is silent or garbled (each also listed in the
design notes):
  R1  sigma ties beyond outdeg go to the lowest original vertex id.
  R2  degrees are the static pattern degrees ("update" re-ranks nothing).
  R3  positions are 0-based: v* takes position 0, the next pick position |R|.
  R4  when the fallback pick has no arc to the placed set, take instead the
      sigma-argmax among unplaced vertices that have an arc (either
      direction) to a placed vertex (keeps every later position anchored).
  R5  if the pattern has no arc pos0->pos1 but has pos1->pos0, a target arc
      (a, b) is tried as the image of pos1->pos0: f(pos0)=b, f(pos1)=a, and
      the validator's checks are mirrored.
  R7  in induced mode the validator also rejects a target arc between the two
      images in the direction where the pattern has none.
  R8  N_x is the set of in- and out-neighbours of x; the test is
      |N_u & N_v| >= |N_0 & N_1|, skipped when the right side is 0.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# Alg. 1
# ---------------------------------------------------------------------------

def _degrees(k, src, dst):
    indeg = [0] * k
    outdeg = [0] * k
    for a, b in zip(src, dst):
        outdeg[int(a)] += 1
        indeg[int(b)] += 1
    return indeg, outdeg


def structural_reorder(k: int, src, dst) -> list[int]:
    """Alg. 1: return pi_inv, the list position -> original pattern vertex."""
    indeg, outdeg = _degrees(k, src, dst)
    total = [indeg[v] + outdeg[v] for v in range(k)]
    arcs = {(int(a), int(b)) for a, b in zip(src, dst)}

    def sigma(v):
        return (total[v], outdeg[v])

    def argmax(cands):
        best = None
        for v in sorted(cands):                      # R1: lowest id wins ties
            if best is None or sigma(v) > sigma(best):
                best = v
        return best

    order = [argmax(range(k))]                       # v* -> position 0 (R3)
    placed = {order[0]}
    while len(placed) < k:
        u = order[-1]                                # last placed vertex
        n_plus = [w for w in range(k) if w not in placed and (u, w) in arcs]
        if n_plus:
            w_star = argmax(n_plus)
        else:
            w_star = argmax([w for w in range(k) if w not in placed])
            if not any((w_star, r) in arcs or (r, w_star) in arcs for r in placed):
                anchored = [w for w in range(k) if w not in placed
                            and any((w, r) in arcs or (r, w) in arcs for r in placed)]
                if anchored:                         # R4
                    w_star = argmax(anchored)
        order.append(w_star)
        placed.add(w_star)
    return order


# ---------------------------------------------------------------------------
# target adjacency for the validators (sorted lists via numpy)
# ---------------------------------------------------------------------------

class TargetLists:
    """Sorted out/in neighbour lists with arc labels, built with numpy lexsort."""

    def __init__(self, n, src, dst, elab):
        src = np.asarray(src, dtype=np.int64)
        dst = np.asarray(dst, dtype=np.int64)
        elab = np.asarray(elab, dtype=np.int64)
        self.n = int(n)
        o = np.lexsort((dst, src))
        self.out_nbr, self.out_lab = dst[o], elab[o]
        self.out_start = np.concatenate([[0], np.cumsum(np.bincount(src, minlength=n))])
        i = np.lexsort((src, dst))
        self.in_nbr, self.in_lab = src[i], elab[i]
        self.in_start = np.concatenate([[0], np.cumsum(np.bincount(dst, minlength=n))])

    def outs(self, v):
        return self.out_nbr[self.out_start[v]:self.out_start[v + 1]]

    def ins(self, v):
        return self.in_nbr[self.in_start[v]:self.in_start[v + 1]]

    def outdeg(self, v):
        return int(self.out_start[v + 1] - self.out_start[v])

    def indeg(self, v):
        return int(self.in_start[v + 1] - self.in_start[v])

    def arc_label(self, a, b):
        """Label of arc (a, b), or None when absent."""
        lst = self.outs(a)
        j = int(np.searchsorted(lst, b))
        if j < lst.shape[0] and lst[j] == b:
            return int(self.out_lab[self.out_start[a] + j])
        return None

    def nbhd(self, v):
        return set(self.outs(v).tolist()) | set(self.ins(v).tolist())


# ---------------------------------------------------------------------------
# the reordered pattern, as the validators see it
# ---------------------------------------------------------------------------

class ReorderedPattern:
    """Pattern after Alg. 1, indexed by position."""

    def __init__(self, pattern):
        k = int(pattern.k)
        self.k = k
        self.order = structural_reorder(k, pattern.src, pattern.dst)
        pos = {v: i for i, v in enumerate(self.order)}
        self.arc = {}
        for a, b, l in zip(pattern.src, pattern.dst, pattern.elab):
            self.arc[(pos[int(a)], pos[int(b)])] = int(l)
        self.vlab = [int(pattern.vlab[v]) for v in self.order]
        self.indeg = [0] * k
        self.outdeg = [0] * k
        for (a, b) in self.arc:
            self.outdeg[a] += 1
            self.indeg[b] += 1

    def nbhd(self, p):
        return {b for (a, b) in self.arc if a == p} | {a for (a, b) in self.arc if b == p}


# ---------------------------------------------------------------------------
# Alg. 2
# ---------------------------------------------------------------------------

def vertex_flags(T: TargetLists, vlab, P: ReorderedPattern) -> np.ndarray:
    """Alg. 2: vertexFlag[v] for every target vertex (for pattern position 0)."""
    vlab = np.asarray(vlab)
    t_in0, t_out0 = P.indeg[0], P.outdeg[0]
    flags = np.zeros(T.n, dtype=bool)
    for v in range(T.n):
        t_in_v, t_out_v = T.indeg(v), T.outdeg(v)
        if vlab[v] == P.vlab[0] and t_in_v >= t_in0 and t_out_v >= t_out0:
            flags[v] = True
    return flags


# ---------------------------------------------------------------------------
# Alg. 3 inside the edge loop of the HiPerMotif algorithm
# ---------------------------------------------------------------------------

def edge_validator(T: TargetLists, vlab, P: ReorderedPattern, induced: bool,
                   a: int, b: int, lab_ab: int, flag_of=None):
    """Try target arc (a, b) as the image of the reordered arc between positions 0 and 1.

    Returns the injected depth-2 state (f(pos0), f(pos1)) or None.  `flag_of`
    gives vertexFlag (Alg. 2); by default it is evaluated on the spot.
    """
    if (0, 1) in P.arc:                   # seed on pos0 -> pos1
        u, v = a, b
        e2, e2r = P.arc[(0, 1)], P.arc.get((1, 0))
    elif (1, 0) in P.arc:                 # R5: seed on pos1 -> pos0
        u, v = b, a
        e2, e2r = P.arc[(1, 0)], None
    else:
        return None
    # vertexFlag[u] and u != v (the loop's guard)
    if flag_of is not None:
        ok_u = flag_of(u)
    else:
        ok_u = (vlab[u] == P.vlab[0] and T.indeg(u) >= P.indeg[0]
                and T.outdeg(u) >= P.outdeg[0])
    if not ok_u or u == v:
        return None
    # match(v, 1)
    if vlab[v] != P.vlab[1]:
        return None
    # match(e1, e2): the seeding arc's label
    if lab_ab != e2:
        return None
    # the other direction between the two images
    if (0, 1) in P.arc:
        back = T.arc_label(v, u)          # e1^r
        if e2r is not None:
            if back is None or back != e2r:
                return None
        elif induced and back is not None:          # R7
            return None
    else:
        fwd = T.arc_label(u, v)           # the pattern has no pos0 -> pos1
        if induced and fwd is not None:             # R7
            return None
    # degree thresholds for position 1
    if not position1_degrees_ok(T, P, v):
        return None
    # neighbour overlap (R8)
    if not overlap_ok(T, P, u, v):
        return None
    return (int(u), int(v))


def position1_degrees_ok(T: TargetLists, P: ReorderedPattern, v: int) -> bool:
    """Alg. 3's degree test on the image of position 1: in- and out-degree at least the pattern's."""
    return T.indeg(v) >= P.indeg[1] and T.outdeg(v) >= P.outdeg[1]


def neighbour_overlap(T: TargetLists, u: int, v: int) -> int:
    """|N_u & N_v|, N_x the set of in- and out-neighbours of x, each counted once (R8)."""
    return len(T.nbhd(u) & T.nbhd(v))


def overlap_ok(T: TargetLists, P: ReorderedPattern, u: int, v: int) -> bool:
    """Alg. 3's neighbour-overlap test |N_u & N_v| >= |N_0 & N_1|, skipped when the right side is 0."""
    need = len(P.nbhd(0) & P.nbhd(1))
    return need == 0 or neighbour_overlap(T, u, v) >= need


def injected_states(graph, pattern, induced: bool) -> np.ndarray:
    """All depth-2 states, as an int32 array [S, 2] of (f(pos0), f(pos1)), sorted."""
    T = TargetLists(graph.n, graph.src, graph.dst, graph.elab)
    P = ReorderedPattern(pattern)
    flags = vertex_flags(T, graph.vlab, P)
    out = []
    for a, b, l in zip(graph.src.tolist(), graph.dst.tolist(), graph.elab.tolist()):
        s = edge_validator(T, graph.vlab, P, induced, a, b, l, flag_of=lambda x: flags[x])
        if s is not None:
            out.append(s)
    return np.array(sorted(out), dtype=np.int32).reshape(-1, 2)
