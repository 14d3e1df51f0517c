"""Pins for the CPU oracle: it is checked against things other than itself.

  * brute force over every injective map (tiny graphs, both modes);
  * hand-worked fixtures (tests/golden/matches_by_hand.txt);
  * closed forms on the complete digraph: n!/(n-k)! monomorphisms for any
    pattern, and for induced matching n!/(n-k)! only when the pattern is
    itself complete, else 0;
  * the labelled directed 3-cycle count equals trace(D0 A0 D1 A0 D2 A0)
    (closed walks; exact int64 matrix products), and the unlabelled count
    equals trace(A^3);
  * embeddings = distinct images x |Aut(P)|, with Aut(P) by brute force;
  * the monomorphism count equals the sum of induced counts over every
    completion of the pattern's non-arcs (k = 3).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import bruteforce
from tests import _golden

MODES = {"mono": oracle.MONO, "induced": oracle.INDUCED}


def _all_weakly_connected_patterns(k):
    pairs = [(i, j) for i in range(k) for j in range(k) if i != j]
    for mask in range(1, 1 << len(pairs)):
        arcs = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        if synth._weakly_connected(k, [a for a, _ in arcs], [b for _, b in arcs]):
            yield arcs


def _pat(k, arcs, vlab, elab, name=""):
    return synth.Pattern(k, np.array([a for a, _ in arcs], np.int32).reshape(-1),
                         np.array([b for _, b in arcs], np.int32).reshape(-1),
                         np.array(vlab, np.int32), np.array(elab, np.int32), name)


# ---------------------------------------------------------------------------
# brute force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(24))
def test_oracle_equals_bruteforce_random(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(4, 8))
    g = synth.small_random_graph(n, p=float(rng.uniform(0.25, 0.7)), n_vlab=int(rng.integers(1, 3)),
                                 n_elab=int(rng.integers(1, 3)), seed=seed,
                                 recip=float(rng.uniform(0, 0.6)), hub=bool(seed % 3 == 0))
    og = oracle.OracleGraph.from_synth(g)
    for t in range(4):
        k = int(rng.integers(2, 5))
        p = synth.random_pattern(rng, k, float(rng.uniform(0.3, 0.9)), n_vlab=int(g.vlab.max()) + 1,
                                 n_elab=int(g.elab.max()) + 1 if g.m else 1)
        for mode in (oracle.MONO, oracle.INDUCED):
            want = bruteforce.matches_of(g, p, induced=bool(mode))
            cnt, rows = og.match(p, mode, threads=3)
            assert cnt == want.shape[0]
            np.testing.assert_array_equal(rows, want)


def test_oracle_equals_bruteforce_all_3vertex_patterns():
    """Every weakly connected 3-vertex digraph (all 54 labelled ones, covering the 13 triad classes)."""
    g = synth.small_random_graph(7, p=0.45, n_vlab=1, n_elab=2, seed=77, recip=0.5)
    og = oracle.OracleGraph.from_synth(g)
    rng = np.random.default_rng(5)
    n_checked = 0
    for arcs in _all_weakly_connected_patterns(3):
        p = _pat(3, arcs, [0, 0, 0], rng.integers(0, 2, len(arcs)))
        for mode in (oracle.MONO, oracle.INDUCED):
            want = bruteforce.matches_of(g, p, induced=bool(mode))
            cnt, rows = og.match(p, mode, threads=2)
            assert cnt == want.shape[0]
            np.testing.assert_array_equal(rows, want)
        n_checked += 1
    assert n_checked == 54


# ---------------------------------------------------------------------------
# hand-worked fixtures
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", _golden.match_cases(), ids=lambda c: c.name)
def test_oracle_hand_worked(case):
    og = oracle.OracleGraph.from_synth(case.graph())
    for mode_name, (count, rows) in case.expect.items():
        cnt, got = og.match(case.pattern(), MODES[mode_name], threads=1)
        assert cnt == count, mode_name
        np.testing.assert_array_equal(got, np.array(rows, np.int32).reshape(-1, case.k))


@pytest.mark.parametrize("case", _golden.match_cases(), ids=lambda c: c.name)
def test_bruteforce_hand_worked(case):
    """The brute force agrees with the hand-derived fixtures too (it pins the oracle elsewhere)."""
    for mode_name, (count, rows) in case.expect.items():
        got = np.asarray(bruteforce.matches_of(case.graph(), case.pattern(), MODES[mode_name]))
        np.testing.assert_array_equal(got.reshape(-1, case.k), np.array(rows, np.int32).reshape(-1, case.k))
        assert got.reshape(-1, case.k).shape[0] == count


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,k", [(5, 2), (6, 3), (7, 3), (6, 4), (8, 4), (7, 5)])
def test_complete_digraph_closed_form(n, k):
    g = synth.complete_digraph(n)
    og = oracle.OracleGraph.from_synth(g)
    rng = np.random.default_rng(n * 10 + k)
    falling = math.perm(n, k)
    for _ in range(3):
        p = synth.random_pattern(rng, k, float(rng.uniform(0.2, 0.8)), n_vlab=1, n_elab=1)
        assert og.match(p, oracle.MONO, rows=False)[0] == falling
        complete = p.mp == k * (k - 1)
        assert og.match(p, oracle.INDUCED, rows=False)[0] == (falling if complete else 0)
    full = _pat(k, [(i, j) for i in range(k) for j in range(k) if i != j], [0] * k,
                [0] * (k * (k - 1)))
    assert og.match(full, oracle.INDUCED, rows=False)[0] == falling
    assert og.match(full, oracle.MONO, rows=False)[0] == falling


def _dense(g, label=None):
    A = np.zeros((g.n, g.n), dtype=np.int64)
    sel = np.ones(g.m, bool) if label is None else (g.elab == label)
    A[g.src[sel], g.dst[sel]] = 1
    return A


def test_labelled_cycle3_trace_identity():
    """Labelled 3-cycle embeddings = trace(D0 A0 D1 A0 D2 A0) on the 1,000-vertex ER workload."""
    g = synth.config1_graph()
    p = synth.config1_pattern()
    A0 = _dense(g, label=0)
    D = [np.diag((g.vlab == i).astype(np.int64)) for i in range(3)]
    want = int(np.trace(D[0] @ A0 @ D[1] @ A0 @ D[2] @ A0))
    og = oracle.OracleGraph.from_synth(g)
    assert og.match(p, oracle.MONO, rows=False)[0] == want
    # the same identity on denser ER graphs, where the count is far from 0
    for seed in (11, 12):
        g2 = synth.er_graph(300, 9000, 3, 2, seed=seed)
        A0 = _dense(g2, label=0)
        D = [np.diag((g2.vlab == i).astype(np.int64)) for i in range(3)]
        want = int(np.trace(D[0] @ A0 @ D[1] @ A0 @ D[2] @ A0))
        got = oracle.OracleGraph.from_synth(g2).match(p, oracle.MONO, rows=False)[0]
        assert got == want and want > 0


def test_unlabelled_cycle3_trace_identity():
    g = synth.config1_graph()
    A = _dense(g)
    want = int(np.trace(A @ A @ A))
    g_u = synth.Graph(g.n, g.src, g.dst, np.zeros(g.n, np.int32), np.zeros(g.m, np.int32))
    p = _pat(3, [(0, 1), (1, 2), (2, 0)], [0, 0, 0], [0, 0, 0])
    got = oracle.OracleGraph.from_synth(g_u).match(p, oracle.MONO, rows=False)[0]
    assert got == want and want > 0


# ---------------------------------------------------------------------------
# automorphism identity
# ---------------------------------------------------------------------------

def _automorphisms(p):
    arcs = {(int(a), int(b)): int(l) for a, b, l in zip(p.src, p.dst, p.elab)}
    out = 0
    for perm in itertools.permutations(range(p.k)):
        if any(p.vlab[perm[i]] != p.vlab[i] for i in range(p.k)):
            continue
        if all(arcs.get((perm[a], perm[b])) == l for (a, b), l in arcs.items()):
            out += 1
    return out


@pytest.mark.parametrize("seed", range(8))
def test_embeddings_equal_images_times_automorphisms(seed):
    rng = np.random.default_rng(300 + seed)
    g = synth.er_graph(40, 500, 2, 2, seed=seed)
    og = oracle.OracleGraph.from_synth(g)
    for _ in range(3):
        k = int(rng.integers(3, 5))
        p = synth.random_pattern(rng, k, float(rng.uniform(0.3, 0.7)), n_vlab=1 + seed % 2,
                                 n_elab=1 + (seed // 2) % 2)
        aut = _automorphisms(p)
        for mode in (oracle.MONO, oracle.INDUCED):
            cnt, rows = og.match(p, mode)
            if mode == oracle.MONO:
                images = {(frozenset(r.tolist()),
                           frozenset((int(r[a]), int(r[b])) for a, b in zip(p.src, p.dst)))
                          for r in rows}
            else:
                images = {frozenset(r.tolist()) for r in rows}
            assert cnt == len(images) * aut


# ---------------------------------------------------------------------------
# monomorphism = sum of induced counts over completions
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_mono_equals_sum_of_induced_completions(seed):
    rng = np.random.default_rng(500 + seed)
    n_elab = 2
    g = synth.er_graph(30, 300, 2, n_elab, seed=40 + seed)
    og = oracle.OracleGraph.from_synth(g)
    k = 3
    p = synth.random_pattern(rng, k, 0.4, n_vlab=2, n_elab=n_elab)
    have = {(int(a), int(b)) for a, b in zip(p.src, p.dst)}
    holes = [(a, b) for a in range(k) for b in range(k) if a != b and (a, b) not in have]
    total = 0
    for choice in itertools.product(range(n_elab + 1), repeat=len(holes)):
        arcs = list(zip(p.src.tolist(), p.dst.tolist()))
        labs = p.elab.tolist()
        for (a, b), c in zip(holes, choice):
            if c:
                arcs.append((a, b))
                labs.append(c - 1)
        q = _pat(k, arcs, p.vlab, labs)
        total += og.match(q, oracle.INDUCED, rows=False)[0]
    assert og.match(p, oracle.MONO, rows=False)[0] == total
    assert total > 0


@pytest.mark.parametrize("seed", range(3))
def test_mono_rows_are_the_disjoint_union_of_induced_completions_k4(seed):
    """Each monomorphism is an induced match of exactly one completion (the one
    that adds the target arcs, with their labels, among the images), so the
    mono rows are the disjoint union of the completions' induced rows."""
    rng = np.random.default_rng(600 + seed)
    g = synth.small_random_graph(14, 0.35, 2, 1, seed=70 + seed, recip=0.4, hub=True)
    og = oracle.OracleGraph.from_synth(g)
    k = 4
    p = synth.random_pattern(rng, k, 0.3, n_vlab=2, n_elab=1)
    have = {(int(a), int(b)) for a, b in zip(p.src, p.dst)}
    holes = [(a, b) for a in range(k) for b in range(k) if a != b and (a, b) not in have]
    parts = []
    for choice in itertools.product((0, 1), repeat=len(holes)):
        arcs = list(zip(p.src.tolist(), p.dst.tolist())) + [h for h, c in zip(holes, choice) if c]
        labs = p.elab.tolist() + [0] * sum(choice)
        parts.append(og.match(_pat(k, arcs, p.vlab, labs), oracle.INDUCED)[1])
    union = np.concatenate(parts).reshape(-1, k)
    mono_c, mono_r = og.match(p, oracle.MONO)
    assert union.shape[0] == mono_c > 0                       # disjoint: no row counted twice
    order = np.lexsort(union.T[::-1])
    np.testing.assert_array_equal(union[order], mono_r)


# ---------------------------------------------------------------------------
# oracle-side sanity: threads and root restriction do not change results
# ---------------------------------------------------------------------------

def test_thread_count_and_root_mask_partition():
    g = synth.er_graph(200, 2400, 2, 2, seed=9)
    og = oracle.OracleGraph.from_synth(g)
    p = _pat(3, [(0, 1), (1, 2), (0, 2)], [0, 1, 0], [0, 0, 1])
    c1, r1 = og.match(p, oracle.MONO, threads=1)
    c8, r8 = og.match(p, oracle.MONO, threads=8)
    assert c1 == c8
    np.testing.assert_array_equal(r1, r8)
    rng = np.random.default_rng(1)
    part = rng.integers(0, 3, g.n)
    parts = [og.match(p, oracle.MONO, root_mask=(part == i).astype(np.uint8)) for i in range(3)]
    assert sum(c for c, _ in parts) == c1
    merged = np.concatenate([r for _, r in parts])
    merged = merged[np.lexsort(merged.T[::-1])]
    np.testing.assert_array_equal(merged, r1)
    for i, (_, r) in enumerate(parts):
        assert np.all(part[r[:, 0]] == i)


def test_oracle_rejects_non_simple_targets():
    with pytest.raises(ValueError):
        oracle.OracleGraph(3, [0, 1], [0, 2], [0, 0, 0], [0, 0])        # self-loop
    with pytest.raises(ValueError):
        oracle.OracleGraph(3, [0, 0], [1, 1], [0, 0, 0], [0, 1])        # duplicate arc


def _induced_subpattern(g, rng, k):
    """The induced subgraph on k vertices of g reached by a randomized search: a
    pattern with at least one induced match (itself)."""
    adj = {v: set() for v in range(g.n)}
    for a, b in zip(g.src, g.dst):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    for _ in range(100):
        seen = [int(rng.integers(0, g.n))]
        while len(seen) < k:
            frontier = sorted({w for v in seen for w in adj[v]} - set(seen))
            if not frontier:
                break
            seen.append(int(rng.choice(frontier)))
        if len(seen) == k:
            break
    idx = {v: i for i, v in enumerate(seen)}
    src, dst, elab = [], [], []
    for a, b, l in zip(g.src, g.dst, g.elab):
        if int(a) in idx and int(b) in idx:
            src.append(idx[int(a)])
            dst.append(idx[int(b)])
            elab.append(int(l))
    return synth.Pattern(k, np.array(src, np.int32), np.array(dst, np.int32),
                         np.array([g.vlab[v] for v in seen], np.int32), np.array(elab, np.int32), f"sub{k}")


@pytest.mark.parametrize("seed", range(6))
def test_oracle_equals_bruteforce_larger_patterns(seed):
    """Patterns of 5 and 6 vertices (the GPU path is compared with the oracle up to 20),
    taken as induced subgraphs of the target so that both modes have matches."""
    rng = np.random.default_rng(2000 + seed)
    g = synth.small_random_graph(7, p=float(rng.uniform(0.3, 0.6)), n_vlab=1 + seed % 2, n_elab=1 + seed % 3 // 2,
                                 seed=50 + seed, recip=0.5, hub=bool(seed % 2))
    og = oracle.OracleGraph.from_synth(g)
    for k in (5, 6):
        p = _induced_subpattern(g, rng, k)
        for mode in (oracle.MONO, oracle.INDUCED):
            want = bruteforce.matches_of(g, p, induced=bool(mode))
            assert want.shape[0] >= 1
            cnt, rows = og.match(p, mode, threads=2)
            assert cnt == want.shape[0]
            np.testing.assert_array_equal(rows, want)
