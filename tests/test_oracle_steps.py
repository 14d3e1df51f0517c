"""Pins for the plain restatements of Alg. 1-3 in oracle/steps.py.

  * Alg. 1 against hand-worked runs (tests/golden/reorder_by_hand.txt) and the
    invariants of the correctness proposition for Alg. 1: the result is a
    permutation, position 0 holds a sigma-argmax, and (with reading R4) every
    later position has an arc to an earlier one.
  * Alg. 2 / Alg. 3 soundness (the validator propositions and the
    completeness theorem for state injection): for every match the oracle
    finds, the pair (f(pos0), f(pos1)) is among the injected states; and every
    injected state is a genuine partial match of positions 0 and 1.
  * Alg. 3's pruning thresholds, which soundness alone cannot pin (a reading
    that under-prunes stays sound): hand-worked injected states
    (tests/golden/states_by_hand.txt) in which the position-1 degree threshold,
    or the neighbour-overlap threshold |N_u & N_v| >= |N_0 & N_1| (R8), alone
    rejects an arc; every planted misreading of either threshold (dropped,
    degrees swapped, only out- or only in-neighbours, a reciprocal neighbour
    counted twice, ">" for ">=") fails one of them.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from oracle import steps
from tests import _golden


@pytest.mark.parametrize("case", _golden.reorder_cases(), ids=lambda c: c["name"])
def test_reorder_hand_worked(case):
    src = [a for a, _ in case["arcs"]]
    dst = [b for _, b in case["arcs"]]
    assert steps.structural_reorder(case["k"], src, dst) == case["order"]


@pytest.mark.parametrize("seed", range(30))
def test_reorder_invariants(seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 12))
    p = synth.random_pattern(rng, k, float(rng.uniform(0.1, 0.7)), n_vlab=1, n_elab=1)
    order = steps.structural_reorder(k, p.src, p.dst)
    assert sorted(order) == list(range(k))
    indeg = np.bincount(p.dst, minlength=k)
    outdeg = np.bincount(p.src, minlength=k)
    sig = [(int(indeg[v] + outdeg[v]), int(outdeg[v])) for v in range(k)]
    assert sig[order[0]] == max(sig)
    arcs = set(zip(p.src.tolist(), p.dst.tolist()))
    for i in range(1, k):
        w = order[i]
        assert any((w, r) in arcs or (r, w) in arcs for r in order[:i])
        last = order[i - 1]
        outs = [x for x in range(k) if (last, x) in arcs and x not in order[:i]]
        if outs:   # the chain rule of Alg. 1: take the best unplaced out-neighbour
            assert w in outs and sig[w] == max(sig[x] for x in outs)


def _graphs():
    yield synth.small_random_graph(9, 0.4, 2, 2, seed=1, recip=0.4, hub=True)
    yield synth.er_graph(60, 900, 2, 2, seed=2)
    yield synth.config2_graph(scale=8)


@pytest.mark.parametrize("gi,g", list(enumerate(_graphs())))
def test_injection_is_sound_and_complete(gi, g):
    og = oracle.OracleGraph.from_synth(g)
    rng = np.random.default_rng(gi)
    T = steps.TargetLists(g.n, g.src, g.dst, g.elab)
    for t in range(6):
        k = int(rng.integers(2, 5))
        p = synth.random_pattern(rng, k, float(rng.uniform(0.3, 0.8)),
                                 n_vlab=int(g.vlab.max()) + 1, n_elab=int(g.elab.max()) + 1)
        P = steps.ReorderedPattern(p)
        for mode in (oracle.MONO, oracle.INDUCED):
            seeds = steps.injected_states(g, p, bool(mode))
            seedset = set(map(tuple, seeds.tolist()))
            assert len(seedset) == seeds.shape[0]
            _, rows = og.match(p, mode)
            for r in rows:                       # completeness
                assert (int(r[P.order[0]]), int(r[P.order[1]])) in seedset
            for u, v in seedset:                 # soundness of each state
                assert g.vlab[u] == P.vlab[0] and g.vlab[v] == P.vlab[1]
                for (a, b), lab in P.arc.items():
                    if {a, b} == {0, 1}:
                        x, y = (u, v) if a == 0 else (v, u)
                        assert T.arc_label(x, y) == lab
                if mode == oracle.INDUCED:
                    if (0, 1) not in P.arc:
                        assert T.arc_label(u, v) is None
                    if (1, 0) not in P.arc:
                        assert T.arc_label(v, u) is None


def test_vertex_flags_hand_case():
    # target: 0->1, 0->2, 3->0, 1->2; labels (0,0,1,0)
    g = synth.Graph(4, np.array([0, 0, 3, 1], np.int32), np.array([1, 2, 0, 2], np.int32),
                    np.array([0, 0, 1, 0], np.int32), np.zeros(4, np.int32))
    T = steps.TargetLists(g.n, g.src, g.dst, g.elab)
    # pattern: out-star 0->1, 0->2 (pos0 = 0 with in 0 / out 2), label 0
    p = synth.Pattern(3, np.array([0, 0], np.int32), np.array([1, 2], np.int32),
                      np.array([0, 0, 0], np.int32), np.zeros(2, np.int32))
    P = steps.ReorderedPattern(p)
    assert P.order[0] == 0
    # only vertex 0 has label 0 and out-degree >= 2
    np.testing.assert_array_equal(steps.vertex_flags(T, g.vlab, P), [True, False, False, False])


def test_reversed_seed_direction():
    """R5: the in-star's first two positions are joined only by pos1 -> pos0."""
    p = synth.Pattern(3, np.array([1, 2], np.int32), np.array([0, 0], np.int32),
                      np.zeros(3, np.int32), np.zeros(2, np.int32))
    P = steps.ReorderedPattern(p)
    assert P.order[:2] == [0, 1] and (1, 0) in P.arc and (0, 1) not in P.arc
    g = synth.Graph(3, np.array([1, 2], np.int32), np.array([0, 0], np.int32),
                    np.zeros(3, np.int32), np.zeros(2, np.int32))
    # target arc 1->0 seeds f(pos0)=0, f(pos1)=1; arc 2->0 seeds (0, 2)
    got = steps.injected_states(g, p, induced=False)
    np.testing.assert_array_equal(got, [[0, 1], [0, 2]])


# ---------------------------------------------------------------------------
# hand-worked injected states (tests/golden/states_by_hand.txt): the
# position-1 degree threshold and the neighbour-overlap threshold of Alg. 3
# each decide some arc on their own
# ---------------------------------------------------------------------------

_STATE_CASES = _golden.match_cases("states_by_hand.txt")


@pytest.mark.parametrize("mode", ["mono", "induced"])
@pytest.mark.parametrize("case", _STATE_CASES, ids=lambda c: c.name)
def test_injected_states_hand_worked(case, mode):
    want = np.array(case.expect[mode][1], np.int32).reshape(-1, 2)
    got = steps.injected_states(case.graph(), case.pattern(), mode == "induced")
    np.testing.assert_array_equal(got, want)


def _fixtures_pass() -> bool:
    for case in _STATE_CASES:
        for mode in ("mono", "induced"):
            want = np.array(case.expect[mode][1], np.int32).reshape(-1, 2)
            got = steps.injected_states(case.graph(), case.pattern(), mode == "induced")
            if not np.array_equal(got, want):
                return False
    return True


def _overlap_out_only(T, u, v):
    return len(set(T.outs(u).tolist()) & set(T.outs(v).tolist()))


def _overlap_in_only(T, u, v):
    return len(set(T.ins(u).tolist()) & set(T.ins(v).tolist()))


def _overlap_repeats_counted(T, u, v):
    # walks u's out-list and then its in-list, so a reciprocal neighbour counts twice
    nv = T.nbhd(v)
    return sum(1 for w in list(T.outs(u)) + list(T.ins(u)) if int(w) in nv)


def _overlap_strict(T, P, u, v):
    need = len(P.nbhd(0) & P.nbhd(1))
    return need == 0 or steps.neighbour_overlap(T, u, v) > need


def _degrees_swapped(T, P, v):
    return T.indeg(v) >= P.outdeg[1] and T.outdeg(v) >= P.indeg[1]


def _degrees_out_only(T, P, v):
    return T.outdeg(v) >= P.outdeg[1]


VALIDATOR_MISTAKES = {
    "drop_position1_degrees": ("position1_degrees_ok", lambda T, P, v: True),
    "position1_degrees_swapped": ("position1_degrees_ok", _degrees_swapped),
    "position1_out_degree_only": ("position1_degrees_ok", _degrees_out_only),
    "drop_overlap": ("overlap_ok", lambda T, P, u, v: True),
    "overlap_strictly_greater": ("overlap_ok", _overlap_strict),
    "overlap_out_neighbours_only": ("neighbour_overlap", _overlap_out_only),
    "overlap_in_neighbours_only": ("neighbour_overlap", _overlap_in_only),
    "overlap_counts_repeats": ("neighbour_overlap", _overlap_repeats_counted),
}


def test_unmutated_validator_passes_fixtures():
    assert _fixtures_pass()


@pytest.mark.parametrize("name", sorted(VALIDATOR_MISTAKES))
def test_planted_validator_mistake_is_caught(monkeypatch, name):
    """Each plausible misreading of Alg. 3's two thresholds fails a hand-worked fixture."""
    attr, wrong = VALIDATOR_MISTAKES[name]
    monkeypatch.setattr(steps, attr, wrong)
    assert not _fixtures_pass()
