"""Batched matching: many patterns in one edge scan and one persistent launch.

Every pattern's result from hm_count_batch / hm_enumerate_batch must equal the
oracle's (and the single-pattern entry points'), bit for bit, whatever else is
in the batch.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2507_04130_gb300 as mod
    assert torch.cuda.is_available()
    mod.set_budget(60_000, 0)
    return mod


def _patterns(rng, count, n_vlab, n_elab, kmin=2, kmax=6):
    return [synth.random_pattern(rng, int(rng.integers(kmin, kmax + 1)), float(rng.uniform(0.3, 1.0)),
                                 n_vlab=n_vlab, n_elab=n_elab, name=f"b{i}") for i in range(count)]


@pytest.mark.parametrize("seed", range(3))
def test_batch_equals_oracle_on_small_graphs(hm, seed):
    rng = np.random.default_rng(70 + seed)
    g = synth.small_random_graph(40, 0.25, 2, 2, seed=seed, recip=0.5, hub=True)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    pats = _patterns(rng, 24, 2, 2)
    modes = [int(x) for x in rng.integers(0, 2, len(pats))]
    P = [hm.Pattern.from_synth(p) for p in pats]
    counts = hm.count_batch(G, P, modes)
    rows = hm.enumerate_batch(G, P, modes)
    for sp, mode, c, r in zip(pats, modes, counts, rows):
        want_c, want_r = og.match(sp, mode)
        assert c == want_c
        np.testing.assert_array_equal(r.cpu().numpy(), want_r)


def test_batch_equals_single_calls_on_rmat(hm):
    g = synth.config2_graph(scale=13)
    G = hm.Graph.from_synth(g)
    pats = synth.config4_patterns(count=96)
    P = [hm.Pattern.from_synth(p) for p in pats]
    counts = hm.count_batch(G, P, hm.INDUCED)
    single = [hm.count_matches(G, p, hm.INDUCED) for p in P]
    assert counts == single
    assert sum(counts) > 0
    rows = hm.enumerate_batch(G, P, hm.INDUCED, counts=counts)
    for p, c, r in zip(P, counts, rows):
        assert r.shape == (c, p.k)
        np.testing.assert_array_equal(r.cpu().numpy(), hm.enumerate_matches(G, p, hm.INDUCED).cpu().numpy())


def test_batch_mixed_modes_duplicates_and_overlap_tests(hm):
    g = synth.er_graph(300, 6000, 2, 2, seed=21)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    tri = synth.Pattern(3, np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32),
                        np.array([0, 1, 0], np.int32), np.array([0, 1, 1], np.int32), "tri")
    arc = synth.Pattern(2, np.array([0], np.int32), np.array([1], np.int32),
                        np.array([1, 0], np.int32), np.array([1], np.int32), "arc")
    star = synth.Pattern(4, np.array([1, 2, 3], np.int32), np.array([0, 0, 0], np.int32),
                         np.zeros(4, np.int32), np.zeros(3, np.int32), "instar")
    pats = [tri, arc, star, tri, arc, star]
    modes = [0, 0, 0, 1, 1, 1]
    P = [hm.Pattern.from_synth(p) for p in pats]
    counts = hm.count_batch(G, P, modes)
    for sp, mode, c in zip(pats, modes, counts):
        assert c == og.match(sp, mode, rows=False)[0]
    rows = hm.enumerate_batch(G, P, modes, counts=counts)
    for sp, mode, r in zip(pats, modes, rows):
        np.testing.assert_array_equal(r.cpu().numpy(), og.match(sp, mode)[1])


def test_batch_capacity_and_empty(hm):
    import ctypes

    g = synth.er_graph(200, 3000, 1, 1, seed=4)
    G = hm.Graph.from_synth(g)
    p = hm.Pattern(3, [0, 1], [1, 2], [0, 0, 0], [0, 0])
    assert hm.count_batch(G, [], []) == []
    counts = hm.count_batch(G, [p, p], hm.MONO)
    assert counts[0] == counts[1] > 5
    handles = (ctypes.c_void_p * 2)(p.handle.value, p.handle.value)
    modes = np.zeros(2, np.int32)
    offs = np.array([0, 3 * 5, 3 * 5 + 3 * counts[1]], np.uint64)      # first region too small
    buf = torch.empty(int(offs[-1]), dtype=torch.int32, device="cuda")
    got = np.zeros(2, np.uint64)
    st = hm.lib.hm_enumerate_batch(G.handle, ctypes.cast(handles, ctypes.c_void_p),
                                   ctypes.c_void_p(modes.ctypes.data), 2, ctypes.c_void_p(buf.data_ptr()),
                                   ctypes.c_void_p(offs.ctypes.data), ctypes.c_void_p(got.ctypes.data),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == hm.binding.HM_ERR_CAPACITY
    assert got.tolist() == counts


def test_autotune_picks_valid_knobs_and_keeps_results(hm):
    g = synth.config2_graph(scale=12)
    G = hm.Graph.from_synth(g)
    pats = synth.config4_patterns(count=32)
    P = [hm.Pattern.from_synth(p) for p in pats]
    ref = hm.count_batch(G, P, hm.INDUCED)
    try:
        best = hm.autotune(G, P, hm.INDUCED, budget_ms=3000)
        assert best["extend_min_blocks"] in (4, 5, 6) and best["ms"] > 0 and not best["from_cache"]
        assert best["warps_per_state"] in (0, 1, 2, 4) and 1 <= best["seeds_per_fetch"] <= 64
        assert hm.get_tuning() == {k: v for k, v in best.items() if k not in ("ms", "from_cache")}
        assert hm.count_batch(G, P, hm.INDUCED) == ref
    finally:
        hm.set_tuning()


def test_autotune_cache_reuses_the_choice_per_graph_and_mix(hm, tmp_path):
    g = synth.config2_graph(scale=11)
    G = hm.Graph.from_synth(g)
    pats = synth.config4_patterns(count=16)
    P = [hm.Pattern.from_synth(p) for p in pats]
    cache = str(tmp_path / "tune.txt")
    try:
        first = hm.autotune(G, P, hm.INDUCED, budget_ms=1500, cache=cache)
        assert not first["from_cache"]
        hm.set_tuning()
        again = hm.autotune(G, P, hm.INDUCED, budget_ms=1500, cache=cache)
        assert again["from_cache"]
        strip = lambda d: {k: v for k, v in d.items() if k not in ("ms", "from_cache")}
        assert strip(again) == strip(first) == hm.get_tuning()
        # another pattern mix is another key: tuned afresh and appended
        other = hm.autotune(G, P[:8], hm.INDUCED, budget_ms=800, cache=cache)
        assert not other["from_cache"]
        assert len(open(cache).read().splitlines()) == 2
    finally:
        hm.set_tuning()
