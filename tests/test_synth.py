"""The seeded input generators: simple digraphs of the stated sizes and shapes.

These check the recipes (sizes, simplicity, label ranges, reciprocity, the
alias sampler's distribution), not the matcher.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth


def _simple(g):
    assert g.src.dtype == np.int32 and g.dst.dtype == np.int32
    assert np.all(g.src != g.dst)
    keys = g.src.astype(np.int64) * g.n + g.dst
    assert np.unique(keys).shape[0] == g.m
    assert g.src.min() >= 0 and g.src.max() < g.n and g.dst.max() < g.n


def test_er_exact_size_and_labels():
    g = synth.er_graph(500, 7000, 4, 3, seed=0)
    _simple(g)
    assert g.m == 7000
    assert set(np.unique(g.vlab)) <= set(range(4)) and set(np.unique(g.elab)) <= set(range(3))


def test_rmat_simple_and_skewed():
    g = synth.config2_graph(scale=12)
    _simple(g)
    deg = np.bincount(g.src, minlength=g.n)
    assert deg.max() > 20 * deg.mean()          # power-law hubs
    assert g.vlab.max() < 8 and g.elab.max() < 4


def test_alias_sampler_matches_weights():
    rng = np.random.default_rng(0)
    w = np.array([1.0, 7.0, 2.0, 0.5, 9.5, 3.0, 0.0, 1.0])
    table = synth._alias_table(w)
    draws = synth._alias_draw(rng, table, 400_000)
    freq = np.bincount(draws, minlength=w.size) / draws.size
    np.testing.assert_allclose(freq, w / w.sum(), atol=3e-3)
    assert freq[6] == 0.0


@pytest.mark.parametrize("recip", [0, 2000])
def test_chung_lu_sizes_and_reciprocity(recip):
    n_unique = 40_000
    g = synth.chung_lu_graph(4000, 2.1, 10, 600, n_unique, recip, synth.CELL_TYPE_WEIGHTS, 3, seed=1)
    _simple(g)
    assert n_unique <= g.m <= n_unique + recip
    keys = g.src.astype(np.int64) * g.n + g.dst
    rev = g.dst.astype(np.int64) * g.n + g.src
    in_pairs = np.isin(rev, keys).mean()
    if recip == 0:
        assert in_pairs < 0.05                     # only chance reciprocity among hubs
    else:
        assert in_pairs >= 2 * (g.m - n_unique) / g.m
    assert g.vlab.max() < 6 and g.elab.max() < 3
    # same seed, same graph
    g2 = synth.chung_lu_graph(4000, 2.1, 10, 600, n_unique, recip, synth.CELL_TYPE_WEIGHTS, 3, seed=1)
    np.testing.assert_array_equal(g.src, g2.src)
    np.testing.assert_array_equal(g.elab, g2.elab)


def test_pattern_recipes():
    b = synth.config4_patterns()
    assert len(b) == 256
    assert {p.k for p in b} <= set(range(3, 7)) and len({p.k for p in b}) == 4
    for p in b:
        assert synth._weakly_connected(p.k, p.src, p.dst)
        assert p.vlab.max() < 8 and (p.elab.max() < 4 if p.mp else True)
        pairs = set(zip(p.src.tolist(), p.dst.tolist()))
        assert len(pairs) == p.mp and all(a != c for a, c in pairs)   # simple
    c = synth.config3_patterns()
    assert len(c) == 5 and all(p.k == 5 and 10 <= p.mp <= 16 for p in c)
    arr = synth.config5_arrivals(100.0, 50)
    times = [t for t, _, _ in arr]
    assert all(b2 > a2 for a2, b2 in zip(times, times[1:]))
    assert {m for _, _, m in arr} == {0, 1}
    assert all(3 <= p.k <= 7 and synth._weakly_connected(p.k, p.src, p.dst) for _, p, _ in arr)
    m = synth.config2_patterns()
    assert [p.name for p in m] == ["ffl_out", "bifan", "cycle4"]
    assert all(p.k == 4 and p.mp == 4 and p.vlab.tolist() == [0, 1, 0, 1] for p in m)


def test_cache_round_trip_and_version_key(tmp_path, monkeypatch):
    monkeypatch.setenv("HM_CACHE", str(tmp_path))
    calls = []

    def gen(n, m, seed=0):
        calls.append(seed)
        return synth.er_graph(n, m, 2, 2, seed=seed)

    g1 = synth.cached("er", gen, 50, 300, seed=4)
    g2 = synth.cached("er", gen, 50, 300, seed=4)          # from the file
    assert calls == [4]
    for a in ("src", "dst", "vlab", "elab"):
        np.testing.assert_array_equal(getattr(g1, a), getattr(g2, a))
    assert g2.n == g1.n and g2.src.dtype == np.int32
    synth.cached("er", gen, 50, 300, seed=5)               # other arguments: generated again
    monkeypatch.setattr(synth, "_GENERATOR_VERSION", synth._GENERATOR_VERSION + 1)
    synth.cached("er", gen, 50, 300, seed=4)               # a new generator version: not reused
    assert calls == [4, 5, 4]
    assert not [p for p in tmp_path.iterdir() if ".tmp" in p.name]
