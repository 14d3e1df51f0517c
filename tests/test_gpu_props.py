"""Multi-property labels and patterns of up to 20 vertices.

* A graph loaded with several properties per vertex and per arc must give
  exactly the matches of the same graph with each distinct property tuple
  replaced by one integer (an encoding built independently here with a dict);
  a pattern tuple the graph lacks matches nothing.
* Patterns of 10-20 vertices (the paper evaluates patterns of 3 to 20 nodes)
  against the oracle.
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


def _encode(rows, table):
    out = []
    for r in map(tuple, rows):
        if r not in table:
            table[r] = len(table) + 1000
        out.append(table[r])
    return np.array(out, np.int32)


@pytest.mark.parametrize("seed", range(3))
def test_property_tuples_equal_their_integer_encoding(hm, seed):
    rng = np.random.default_rng(900 + seed)
    g = synth.er_graph(500, 8000, 1, 1, seed=seed)
    vprops = rng.integers(-2, 2, size=(g.n, 2)).astype(np.int32)
    eprops = rng.integers(0, 2, size=(g.m, 3)).astype(np.int32)
    G = hm.Graph.with_properties(g.n, g.src, g.dst, vprops, eprops)
    vt, et = {}, {}
    ge = synth.Graph(g.n, g.src, g.dst, _encode(vprops, vt), _encode(eprops, et))
    og = oracle.OracleGraph.from_synth(ge)
    for t in range(6):
        k = int(rng.integers(2, 6))
        p = synth.random_pattern(rng, k, float(rng.uniform(0.3, 0.8)), n_vlab=1, n_elab=1)
        pv = vprops[rng.integers(0, g.n, k)]
        pe = eprops[rng.integers(0, g.m, p.mp)]
        if t == 5:  # a tuple the graph does not have
            pv = pv.copy()
            pv[0] = (7, 7)
        P = hm.Pattern.with_properties(G, p.k, p.src, p.dst, pv, pe)
        pe_enc = synth.Pattern(k, p.src, p.dst, _encode(pv, dict(vt)), _encode(pe, dict(et)))
        for mode in (hm.MONO, hm.INDUCED):
            want_c, want_r = og.match(pe_enc, mode)
            assert hm.count_matches(G, P, mode) == want_c
            np.testing.assert_array_equal(hm.enumerate_matches(G, P, mode).cpu().numpy(), want_r)
            if t == 5:
                assert want_c == 0


def test_props_api_errors(hm):
    g = synth.er_graph(50, 200, 1, 1, seed=1)
    G = hm.Graph.from_synth(g)           # loaded without properties
    with pytest.raises(hm.HMError):
        hm.Pattern.with_properties(G, 2, [0], [1], [[0], [0]], [[0]])


def _path(k, rng, n_vlab):
    return synth.Pattern(k, np.arange(k - 1, dtype=np.int32), np.arange(1, k, dtype=np.int32),
                         rng.integers(0, n_vlab, k).astype(np.int32), np.zeros(k - 1, np.int32),
                         f"path{k}")


@pytest.mark.parametrize("k", [10, 14, 20])
def test_large_patterns_against_the_oracle(hm, k):
    rng = np.random.default_rng(k)
    g = synth.er_graph(300, 2400, 6, 1, seed=k)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    pats = [_path(k, rng, 6)]
    # two random trees with random arc directions
    for _ in range(2):
        src, dst = [], []
        for v in range(1, k):
            u = int(rng.integers(0, v))
            if rng.random() < 0.5:
                src.append(u); dst.append(v)
            else:
                src.append(v); dst.append(u)
        pats.append(synth.Pattern(k, np.array(src, np.int32), np.array(dst, np.int32),
                                  rng.integers(0, 6, k).astype(np.int32), np.zeros(k - 1, np.int32),
                                  f"tree{k}"))
    for sp in pats:
        P = hm.Pattern.from_synth(sp)
        for mode in (hm.MONO, hm.INDUCED):
            want_c, want_r = og.match(sp, mode)
            assert hm.count_matches(G, P, mode) == want_c
            np.testing.assert_array_equal(hm.enumerate_matches(G, P, mode).cpu().numpy(), want_r)
