"""GPU parity: the CUDA path against the CPU oracle, bit-exact (integer work).

Counts and the sorted row lists must be identical; the intermediate results
(built adjacency, injected depth-2 states) are checked against plain
restatements (numpy sort, oracle/steps.py).  All calls go through the C ABI.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import steps
from tests import _golden

pytestmark = pytest.mark.gpu

MODES = (oracle.MONO, oracle.INDUCED)


@pytest.fixture(scope="module")
def hm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2507_04130_gb300 as mod
    assert torch.cuda.is_available()
    mod.set_budget(60_000, 0)
    return mod


def _check(hm, G, og, sp, mode, rows=True):
    P = hm.Pattern.from_synth(sp)
    want_count, want_rows = og.match(sp, mode, rows=rows)
    got = hm.count_matches(G, P, mode)
    assert got == want_count, (sp.name, mode, got, want_count)
    if rows:
        r = hm.enumerate_matches(G, P, mode).cpu().numpy()
        assert r.shape == want_rows.shape
        np.testing.assert_array_equal(r, want_rows)
    return want_count


# ---------------------------------------------------------------------------
# graph build
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_graph_build_matches_numpy_sort(hm, seed):
    g = synth.er_graph(3000 + 517 * seed, 40000 + 999 * seed, 4, 5, seed=seed)
    for device in (False, True):
        G = hm.Graph.from_synth(g, device=device)
        ex = G.export()
        o = np.lexsort((g.dst, g.src))
        np.testing.assert_array_equal(ex["out_adj"], g.dst[o])
        np.testing.assert_array_equal(ex["out_elab"], g.elab[o])
        np.testing.assert_array_equal(ex["out_off"], np.concatenate([[0], np.cumsum(np.bincount(g.src, minlength=g.n))]))
        i = np.lexsort((g.src, g.dst))
        np.testing.assert_array_equal(ex["in_adj"], g.src[i])
        np.testing.assert_array_equal(ex["in_elab"], g.elab[i])
        np.testing.assert_array_equal(ex["in_off"], np.concatenate([[0], np.cumsum(np.bincount(g.dst, minlength=g.n))]))


def test_graph_build_rmat_hubs(hm):
    g = synth.config2_graph(scale=14)
    ex = hm.Graph.from_synth(g).export()
    o = np.lexsort((g.dst, g.src))
    np.testing.assert_array_equal(ex["out_adj"], g.dst[o])
    np.testing.assert_array_equal(ex["out_elab"], g.elab[o])


def _export_groups(hm, G):
    import ctypes
    n, m = G.n, G.m
    nd = np.zeros(2, np.int64)
    hm.check(hm.lib.hm_graph_export_groups(G.handle, None, None, None, None, None,
                                           ctypes.c_void_p(nd.ctypes.data)), "groups")
    out = {"gout": np.zeros(max(m, 1), np.int32), "gin": np.zeros(max(m, 1), np.int32),
           "vdir": np.zeros((max(n, 1), 4), np.int32),
           "dout": np.zeros((max(int(nd[0]), 1), 4), np.int32),
           "din": np.zeros((max(int(nd[1]), 1), 4), np.int32)}
    hm.check(hm.lib.hm_graph_export_groups(G.handle, *[ctypes.c_void_p(out[k].ctypes.data) for k in
                                                       ("gout", "gin", "vdir", "dout", "din")],
                                           None), "groups")
    return out, nd


@pytest.mark.parametrize("big", [False, True], ids=["rmat10", "er400k"])
@pytest.mark.parametrize("signed_labels", [False, True])
def test_label_grouped_lists_and_directory(hm, signed_labels, big):
    # er400k: more than 2^18 arcs, so the build's row sorts run as one
    # cooperative launch, with 13-bit vertex ids and 2-3-bit labels whose
    # digits span several key columns
    g = synth.er_graph(6000, 400_000, 3, 5, seed=11) if big else synth.config2_graph(scale=10)
    if big:
        ex0 = hm.Graph.from_synth(g).export()
        o = np.lexsort((g.dst, g.src))
        np.testing.assert_array_equal(ex0["out_adj"], g.dst[o])
        np.testing.assert_array_equal(ex0["out_elab"], g.elab[o])
        i = np.lexsort((g.src, g.dst))
        np.testing.assert_array_equal(ex0["in_adj"], g.src[i])
    if signed_labels:   # labels outside [0, 2^24) take the 32-bit key path
        g = synth.Graph(g.n, g.src, g.dst, (g.vlab * 1000003 - 5).astype(np.int32),
                        (g.elab * -7).astype(np.int32))
    G = hm.Graph.from_synth(g)
    ex = G.export()
    gr, nd = _export_groups(hm, G)
    for side, key, other, off in (("out", g.src, g.dst, ex["out_off"]), ("in", g.dst, g.src, ex["in_off"])):
        o = np.lexsort((other, g.vlab[other], g.elab, key))
        glist = gr["gout" if side == "out" else "gin"][: g.m]
        np.testing.assert_array_equal(glist, other[o])
        ks, el, vl = key[o], g.elab[o], g.vlab[other][o]
        starts = np.flatnonzero(np.r_[True, (ks[1:] != ks[:-1]) | (el[1:] != el[:-1]) | (vl[1:] != vl[:-1])])
        ends = np.r_[starts[1:], g.m]
        d = gr["dout" if side == "out" else "din"][: starts.shape[0]]
        assert int(nd[0 if side == "out" else 1]) == starts.shape[0]
        np.testing.assert_array_equal(d[:, 0], el[starts])
        np.testing.assert_array_equal(d[:, 1], vl[starts])
        np.testing.assert_array_equal(d[:, 2], starts - off[ks[starts]])
        np.testing.assert_array_equal(d[:, 3], ends - off[ks[starts]])
        col = 0 if side == "out" else 2
        first = np.searchsorted(starts, off[:-1])
        cnt = np.searchsorted(starts, off[1:]) - first
        np.testing.assert_array_equal(gr["vdir"][: g.n, col], first)
        np.testing.assert_array_equal(gr["vdir"][: g.n, col + 1], cnt)


def test_graph_build_edge_cases(hm):
    G = hm.Graph(5, [], [], [0] * 5, [])            # no arcs
    ex = G.export()
    assert ex["out_off"].tolist() == [0] * 6 and ex["in_off"].tolist() == [0] * 6
    G = hm.Graph(0, [], [], [], [])                  # empty graph
    assert G.n == 0
    G = hm.Graph(4, [3], [0], [1, 2, 3, 4], [9])      # isolated vertices around one arc
    ex = G.export()
    assert ex["out_off"].tolist() == [0, 0, 0, 0, 1]
    assert ex["in_off"].tolist() == [0, 1, 1, 1, 1]
    for src, dst, status in ([[0, 1], [1, 1], "HM_ERR_SELF_LOOP"],
                             [[0, 0], [1, 1], "HM_ERR_DUP_EDGE"],
                             [[0, 7], [1, 2], "HM_ERR_ARG"]):
        with pytest.raises(hm.HMError) as ei:
            hm.Graph(3, src, dst, [0, 0, 0], [0] * len(src))
        assert ei.value.status == getattr(hm.binding, status)


# ---------------------------------------------------------------------------
# injected states (Alg. 2 + Alg. 3 inside the edge loop)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_injected_states_equal_plain_validators(hm, seed):
    rng = np.random.default_rng(seed)
    g = synth.er_graph(300, 6000, 2, 2, seed=100 + seed) if seed % 2 else \
        synth.small_random_graph(40, 0.3, 2, 2, seed=seed, recip=0.5, hub=True)
    G = hm.Graph.from_synth(g)
    for t in range(6):
        k = int(rng.integers(2, 6))
        sp = synth.random_pattern(rng, k, float(rng.uniform(0.3, 0.9)), n_vlab=2, n_elab=2)
        P = hm.Pattern.from_synth(sp)
        for mode in MODES:
            want = steps.injected_states(g, sp, bool(mode))
            got = hm.injected_states(G, P, mode).cpu().numpy()
            got = got[np.lexsort((got[:, 1], got[:, 0]))] if got.shape[0] else got.reshape(0, 2)
            np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("case", _golden.match_cases("states_by_hand.txt"), ids=lambda c: c.name)
def test_injected_states_hand_worked(hm, case):
    """The hand-worked states in which the position-1 degree threshold or the
    neighbour-overlap threshold alone rejects an arc (Alg. 3, reading R8)."""
    G = hm.Graph.from_synth(case.graph())
    P = hm.Pattern.from_synth(case.pattern())
    for mode_name, (_, states) in case.expect.items():
        mode = oracle.MONO if mode_name == "mono" else oracle.INDUCED
        got = hm.injected_states(G, P, mode).cpu().numpy().reshape(-1, 2)
        got = got[np.lexsort((got[:, 1], got[:, 0]))]
        np.testing.assert_array_equal(got, np.array(states, np.int32).reshape(-1, 2))


# ---------------------------------------------------------------------------
# full matching, small and medium inputs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", _golden.match_cases(), ids=lambda c: c.name)
def test_hand_worked(hm, case):
    G = hm.Graph.from_synth(case.graph())
    P = hm.Pattern.from_synth(case.pattern())
    for mode_name, (count, rows) in case.expect.items():
        mode = oracle.MONO if mode_name == "mono" else oracle.INDUCED
        assert hm.count_matches(G, P, mode) == count
        got = hm.enumerate_matches(G, P, mode).cpu().numpy()
        np.testing.assert_array_equal(got, np.array(rows, np.int32).reshape(-1, case.k))


@pytest.mark.parametrize("seed", range(12))
def test_random_small_graphs(hm, seed):
    rng = np.random.default_rng(2000 + seed)
    g = synth.small_random_graph(int(rng.integers(6, 40)), float(rng.uniform(0.1, 0.6)),
                                 int(rng.integers(1, 3)), int(rng.integers(1, 3)), seed=seed,
                                 recip=float(rng.uniform(0, 0.7)), hub=seed % 2 == 0)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    for t in range(8):
        k = int(rng.integers(2, 7))
        sp = synth.random_pattern(rng, k, float(rng.uniform(0.2, 1.0)), n_vlab=int(g.vlab.max()) + 1,
                                  n_elab=int(g.elab.max()) + 1)
        for mode in MODES:
            _check(hm, G, og, sp, mode)


def test_complete_digraph(hm):
    g = synth.complete_digraph(9)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    rng = np.random.default_rng(0)
    for k in (2, 3, 4, 5):
        sp = synth.random_pattern(rng, k, 0.5, n_vlab=1, n_elab=1)
        for mode in MODES:
            _check(hm, G, og, sp, mode)


def test_complete_digraph_large_row_sort(hm):
    """303,600 rows of 5-bit ids: the row sort's single-launch path with digits spanning columns.

    On the complete digraph every injective map is a monomorphism of any
    4-vertex pattern (the closed form n!/(n-k)!), so the sorted rows are
    exactly the ordered 4-permutations of 0..24 in lexicographic order.
    """
    import itertools
    n, k = 25, 4
    G = hm.Graph.from_synth(synth.complete_digraph(n))
    sp = synth.Pattern(k, np.array([0, 1, 2, 3], np.int32), np.array([1, 2, 3, 0], np.int32),
                       np.zeros(k, np.int32), np.zeros(k, np.int32))
    want = np.array(list(itertools.permutations(range(n), k)), np.int32)
    assert want.shape[0] == 303_600 > (1 << 18)
    P = hm.Pattern.from_synth(sp)
    try:
        hm.set_tuning(symmetry=-1)   # every row found by the search, none as an automorphic image
        rows = hm.enumerate_matches(G, P, hm.MONO).cpu().numpy()
    finally:
        hm.set_tuning()
    np.testing.assert_array_equal(rows, want)
    np.testing.assert_array_equal(hm.enumerate_matches(G, P, hm.MONO).cpu().numpy(), want)


def test_er_workload_cycle3(hm):
    """1,000-vertex ER workload: labelled 3-cycle (count + rows) and its unlabelled count."""
    g = synth.config1_graph()
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    sp = synth.config1_pattern()
    for mode in MODES:
        _check(hm, G, og, sp, mode)
    gu = synth.Graph(g.n, g.src, g.dst, np.zeros(g.n, np.int32), np.zeros(g.m, np.int32))
    Gu = hm.Graph.from_synth(gu)
    ogu = oracle.OracleGraph.from_synth(gu)
    spu = synth.Pattern(3, sp.src, sp.dst, np.zeros(3, np.int32), np.zeros(3, np.int32), "cycle3u")
    c = _check(hm, Gu, ogu, spu, oracle.MONO)
    assert c > 0


@pytest.mark.parametrize("scale", [10, 13])
def test_rmat_reduced_three_motifs(hm, scale):
    g = synth.config2_graph(scale=scale)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    for sp in synth.config2_patterns():
        for mode in MODES:
            _check(hm, G, og, sp, mode)


def test_rmat_reduced_random_batch_patterns(hm):
    g = synth.config2_graph(scale=12)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    for sp in synth.config4_patterns(count=40):
        _check(hm, G, og, sp, oracle.INDUCED)
        _check(hm, G, og, sp, oracle.MONO, rows=False)


def test_connectome_reduced(hm):
    g = synth.config3_graph(n=3000, n_unique=120_000, n_recip=6000)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    for sp in synth.config3_patterns():
        _check(hm, G, og, sp, oracle.MONO, rows=False)
        _check(hm, G, og, sp, oracle.INDUCED)


def test_unlabelled_hubs_force_donation(hm):
    """Power-law graph, one label: a few seeds own most of the work, so warps must share it."""
    g0 = synth.config3_graph(n=2000, n_unique=60_000, n_recip=3000)
    g = synth.Graph(g0.n, g0.src, g0.dst, np.zeros(g0.n, np.int32), np.zeros(g0.m, np.int32))
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    sp = synth.Pattern(4, np.array([0, 1, 2], np.int32), np.array([1, 2, 3], np.int32),
                       np.zeros(4, np.int32), np.zeros(3, np.int32), "path4")
    _check(hm, G, og, sp, oracle.MONO, rows=False)
    hm.set_tuning(leaf_flatten=-1)   # one survivor at a time: every range can be split
    try:
        _check(hm, G, og, sp, oracle.MONO, rows=False)
        st = hm.last_stats()
    finally:
        hm.set_tuning()
    assert st["tasks_donated"] > 0


# ---------------------------------------------------------------------------
# API behaviour on the device
# ---------------------------------------------------------------------------

def test_capacity_protocol(hm):
    g = synth.er_graph(200, 3000, 1, 1, seed=5)
    G = hm.Graph.from_synth(g)
    sp = synth.Pattern(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32),
                       np.zeros(3, np.int32), np.zeros(2, np.int32))
    P = hm.Pattern.from_synth(sp)
    total = hm.count_matches(G, P, hm.MONO)
    assert total > 10
    buf = torch.empty(10 * 3, dtype=torch.int32, device="cuda")
    with pytest.raises(hm.HMError) as ei:
        hm.enumerate_matches(G, P, hm.MONO, out=buf, capacity=10)
    assert ei.value.status == hm.binding.HM_ERR_CAPACITY and ei.value.count == total
    rows = hm.enumerate_matches(G, P, hm.MONO, capacity=total)
    assert rows.shape == (total, 3)


def test_budget_watchdog_then_recovery(hm):
    g = synth.er_graph(2000, 60000, 1, 1, seed=6)
    G = hm.Graph.from_synth(g)
    sp = synth.Pattern(4, np.array([0, 1, 2], np.int32), np.array([1, 2, 3], np.int32),
                       np.zeros(4, np.int32), np.zeros(3, np.int32))
    P = hm.Pattern.from_synth(sp)
    full = hm.count_matches(G, P, hm.MONO)
    hm.set_budget(60_000, 64)
    try:
        with pytest.raises(hm.HMError) as ei:
            hm.count_matches(G, P, hm.MONO)
        assert ei.value.status == hm.binding.HM_ERR_BUDGET
    finally:
        hm.set_budget(60_000, 0)
    assert hm.count_matches(G, P, hm.MONO) == full


def test_rooted_counts_partition(hm):
    g = synth.config2_graph(scale=11)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    rng = np.random.default_rng(3)
    for sp in synth.config2_patterns():
        P = hm.Pattern.from_synth(sp)
        total = hm.count_matches(G, P, hm.INDUCED)
        part = rng.integers(0, 3, g.n)
        for root in range(sp.k):
            s = 0
            for i in range(3):
                mask = (part == i).astype(np.uint8)
                c = hm.count_matches_rooted(G, P, hm.INDUCED, root, mask)
                if root == 0:
                    assert c == og.match(sp, oracle.INDUCED, rows=False, root_mask=mask)[0]
                s += c
            assert s == total


def test_empty_and_label_free_results(hm):
    g = synth.er_graph(100, 500, 2, 2, seed=8)
    G = hm.Graph.from_synth(g)
    sp = synth.Pattern(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32),
                       np.array([7, 7, 7], np.int32), np.zeros(2, np.int32))   # label absent
    P = hm.Pattern.from_synth(sp)
    assert hm.count_matches(G, P, hm.MONO) == 0
    assert hm.enumerate_matches(G, P, hm.MONO).shape == (0, 3)
    E = hm.Graph(50, [], [], [0] * 50, [])
    assert hm.count_matches(E, P, hm.MONO) == 0


def test_stream_ordering_on_side_stream(hm):
    g = synth.er_graph(500, 8000, 2, 2, seed=9)
    og = oracle.OracleGraph.from_synth(g)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        G = hm.Graph.from_synth(g, stream=s)
        sp = synth.config1_pattern()
        P = hm.Pattern.from_synth(sp)
        rows = hm.enumerate_matches(G, P, hm.MONO, stream=s)
        host = rows.cpu().numpy()
    np.testing.assert_array_equal(host, og.match(sp, oracle.MONO)[1])


@pytest.mark.parametrize("nparts", [1, 2, 3, 8])
def test_arc_range_parts_partition_the_matches(hm, nparts):
    g = synth.config2_graph(scale=12)
    G = hm.Graph.from_synth(g)
    for sp in synth.config2_patterns():
        P = hm.Pattern.from_synth(sp)
        full = hm.enumerate_matches(G, P, hm.INDUCED).cpu().numpy()
        parts, total = [], 0
        for i in range(nparts):
            c = hm.count_matches_part(G, P, hm.INDUCED, i, nparts)
            buf = torch.empty(max(c, 1) * sp.k, dtype=torch.int32, device="cuda")
            r = hm.enumerate_matches_part(G, P, hm.INDUCED, i, nparts, buf).cpu().numpy()
            assert r.shape[0] == c
            if c > 1:
                assert np.all(np.diff(r[:, 0]) >= 0)
            parts.append(r)
            total += c
        assert total == full.shape[0]
        merged = np.concatenate(parts)
        merged = merged[np.lexsort(merged.T[::-1])]
        np.testing.assert_array_equal(merged, full)
    with pytest.raises(hm.HMError):
        hm.count_matches_part(G, P, hm.INDUCED, nparts, nparts)


def test_instrumented_kernels_agree_and_count_bytes(hm):
    g = synth.config2_graph(scale=12)
    G = hm.Graph.from_synth(g)
    sp = synth.config2_patterns()[1]
    P = hm.Pattern.from_synth(sp)
    plain = hm.enumerate_matches(G, P, hm.INDUCED).cpu().numpy()
    st0 = hm.last_stats()
    assert st0["bytes_extend"] == 0 and st0["kernel_launches"] >= 3
    hm.set_counters(True)
    try:
        inst = hm.enumerate_matches(G, P, hm.INDUCED).cpu().numpy()
        st = hm.last_stats()
    finally:
        hm.set_counters(False)
    np.testing.assert_array_equal(inst, plain)
    assert st["bytes_edge_scan"] >= 12 * g.m
    assert st["bytes_extend"] > 0 and st["candidates"] > 0
    # the cost model: 12 B per arc scanned at least; 8 B per candidate read at least
    assert st["model_bytes_edge_scan"] >= 12 * g.m
    assert st["model_bytes_extend"] >= 8 * st["candidates"]


@pytest.mark.parametrize("knobs", [dict(extend_min_blocks=5), dict(extend_min_blocks=6),
                                   dict(pair_mode=1), dict(split_min=2, seeds_per_fetch=7),
                                   dict(pair_mode=1, split_min=2, poll_every=1),
                                   dict(poll_every=65536), dict(leaf_flatten=-1),
                                   dict(leaf_flatten=-1, pair_mode=1, split_min=2),
                                   dict(split_min=1000, seeds_per_fetch=64),
                                   dict(arc_filter=-1), dict(arc_filter=1),
                                   dict(arc_filter=1, leaf_flatten=-1, pair_mode=1),
                                   dict(warps_per_state=2), dict(warps_per_state=4, seeds_per_fetch=3),
                                   dict(warps_per_state=4, leaf_flatten=-1, split_min=2),
                                   dict(warps_per_state=2, symmetry=-1, arc_filter=-1),
                                   dict(lookahead=1), dict(lookahead=1, pair_mode=1, split_min=2),
                                   dict(lookahead=1, leaf_flatten=-1, warps_per_state=2)])
def test_tuning_knobs_never_change_results(hm, knobs):
    g0 = synth.config3_graph(n=2000, n_unique=60_000, n_recip=3000)
    g = synth.Graph(g0.n, g0.src, g0.dst, (g0.vlab % 2).astype(np.int32), g0.elab % 2)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    rng = np.random.default_rng(17)
    pats = [synth.random_pattern(rng, int(rng.integers(3, 6)), 0.5, n_vlab=2, n_elab=2)
            for _ in range(4)]
    hm.set_tuning(**knobs)
    try:
        for sp in pats:
            _check(hm, G, og, sp, oracle.INDUCED)
            _check(hm, G, og, sp, oracle.MONO, rows=False)
    finally:
        hm.set_tuning()


def test_results_do_not_depend_on_the_order(hm):
    """The reordering is a heuristic: breadth-first order gives the same sorted rows as Alg. 1's."""
    from tests.test_boundary import _bfs_order

    g = synth.config2_graph(scale=12)
    G = hm.Graph.from_synth(g)
    rng = np.random.default_rng(31)
    for _ in range(12):
        sp = synth.random_pattern(rng, int(rng.integers(3, 8)), float(rng.uniform(0.3, 0.8)),
                                  n_vlab=3, n_elab=2)
        P1 = hm.Pattern.from_synth(sp)
        P2 = hm.Pattern.from_synth(sp, order=_bfs_order(sp.k, sp.src, sp.dst))
        for mode in MODES:
            a = hm.enumerate_matches(G, P1, mode).cpu().numpy()
            b = hm.enumerate_matches(G, P2, mode).cpu().numpy()
            np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------------------
# shared position-0 states (position 1 chosen last)
# ---------------------------------------------------------------------------

def _position1_is_pendant(hm, sp):
    """Does the vertex at position 1 of Alg. 1's order touch only the vertex at position 0?"""
    order = hm.Pattern.from_synth(sp).order
    v0, v1 = order[0], order[1]
    nb = {int(b) for a, b in zip(sp.src, sp.dst) if a == v1} | {int(a) for a, b in zip(sp.src, sp.dst) if b == v1}
    return nb == {v0}


def _pendant_patterns(hm, rng, count, n_vlab, n_elab):
    out = []
    for _ in range(20000):
        k = int(rng.integers(3, 7))
        sp = synth.random_pattern(rng, k, float(rng.uniform(0.15, 0.6)), n_vlab=n_vlab, n_elab=n_elab,
                                  name=f"pend{len(out)}")
        if _position1_is_pendant(hm, sp):
            out.append(sp)
            if len(out) == count:
                break
    assert len(out) == count
    return out


def test_ffl_out_has_a_pendant_position_1(hm):
    ffl = synth.config2_patterns()[0]
    assert ffl.name == "ffl_out" and _position1_is_pendant(hm, ffl)


@pytest.mark.parametrize("seed", range(4))
def test_shared_position0_states_equal_the_oracle(hm, seed):
    rng = np.random.default_rng(300 + seed)
    g = synth.small_random_graph(60, 0.2, 2, 2, seed=seed, recip=0.4, hub=True)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    for sp in _pendant_patterns(hm, rng, 6, 2, 2):
        for mode in MODES:
            want_c, want_r = og.match(sp, mode)
            for share in (1, -1):
                hm.set_tuning(share_seeds=share)
                try:
                    P = hm.Pattern.from_synth(sp)
                    assert hm.count_matches(G, P, mode) == want_c, (sp.name, mode, share)
                    np.testing.assert_array_equal(hm.enumerate_matches(G, P, mode).cpu().numpy(), want_r)
                finally:
                    hm.set_tuning()


@pytest.mark.parametrize("knobs", [dict(arc_filter=-1), dict(leaf_flatten=-1), dict(pair_mode=1, split_min=2),
                                   dict(split_min=2, poll_every=1), dict(warps_per_state=4),
                                   dict(warps_per_state=2, seeds_per_fetch=5)])
def test_shared_position0_states_with_other_knobs(hm, knobs):
    g0 = synth.config3_graph(n=2000, n_unique=60_000, n_recip=3000)
    g = synth.Graph(g0.n, g0.src, g0.dst, (g0.vlab % 2).astype(np.int32), g0.elab % 2)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    pats = _pendant_patterns(hm, np.random.default_rng(31), 4, 2, 2)
    hm.set_tuning(**knobs)
    try:
        for sp in pats:
            _check(hm, G, og, sp, oracle.INDUCED)
            _check(hm, G, og, sp, oracle.MONO, rows=False)
    finally:
        hm.set_tuning()


def test_shared_position0_states_rooted_and_parts(hm):
    g = synth.config2_graph(scale=11)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    ffl = synth.config2_patterns()[0]
    P = hm.Pattern.from_synth(ffl)
    rng = np.random.default_rng(8)
    for mode in MODES:
        total = hm.count_matches(G, P, mode)
        assert total == og.match(ffl, mode, rows=False)[0]
        part = rng.integers(0, 3, g.n)
        for root in range(ffl.k):
            s = 0
            for i in range(3):
                mask = (part == i).astype(np.uint8)
                c = hm.count_matches_rooted(G, P, mode, root, mask)
                if root == 0:
                    assert c == og.match(ffl, mode, rows=False, root_mask=mask)[0]
                s += c
            assert s == total
        assert sum(hm.count_matches_part(G, P, mode, i, 3) for i in range(3)) == total


def test_rows_into_an_unaligned_output_buffer(hm):
    """A caller's row buffer need not be 16-byte aligned (the sort then takes its generic path)."""
    g = synth.config2_graph(scale=11)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    sp = synth.config2_patterns()[1]
    P = hm.Pattern.from_synth(sp)
    want_c, want_r = og.match(sp, oracle.INDUCED)
    assert want_c > 1
    big = torch.empty(want_c * sp.k + 1, dtype=torch.int32, device="cuda")
    out = big[1:]                       # 4-byte offset
    assert out.data_ptr() % 16 != 0
    rows = hm.enumerate_matches(G, P, hm.INDUCED, out=out, capacity=want_c)
    np.testing.assert_array_equal(rows.cpu().numpy(), want_r)
