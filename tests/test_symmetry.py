"""Symmetry breaking: the same matches as searching every map for itself.

The matches of a pattern (Sec. II-A, Eqs. 1-3) fall into orbits of exactly
|Aut| maps under the pattern's label-preserving automorphisms (the oracle's
own tests pin embeddings = images x |Aut| by brute force).  The library
searches one map per orbit and emits its |Aut| images, so

  * the automorphism group it uses (hm_pattern_automorphisms) must be the
    full group, checked against a plain enumeration of every permutation
    (CPU, no device);
  * counts and sorted rows must equal the oracle's with symmetry breaking on
    and off, single and batched, on symmetric patterns in both modes (GPU).
"""
from __future__ import annotations

import ctypes
import itertools

import numpy as np
import pytest
import torch

import oracle
import synth


@pytest.fixture(scope="module")
def hm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2507_04130_gb300 as mod
    return mod


def _brute_aut(p) -> int:
    arcs = {(int(a), int(b)): int(l) for a, b, l in zip(p.src, p.dst, p.elab)}
    n = 0
    for perm in itertools.permutations(range(p.k)):
        if any(p.vlab[perm[i]] != p.vlab[i] for i in range(p.k)):
            continue
        if all(arcs.get((perm[a], perm[b])) == l for (a, b), l in arcs.items()):
            n += 1
    return n


def _pat(k, arcs, vlab=None, elab=None, name=""):
    a = np.array(arcs, np.int32).reshape(-1, 2)
    return synth.Pattern(k, a[:, 0].copy(), a[:, 1].copy(),
                         np.array(vlab if vlab is not None else [0] * k, np.int32),
                         np.array(elab if elab is not None else [0] * len(arcs), np.int32), name)


def _cycle(k, vlab=None):
    return _pat(k, [(i, (i + 1) % k) for i in range(k)], vlab,
                name=f"cycle{k}" + ("_" + "".join(map(str, vlab)) if vlab else ""))


SYMMETRIC = [
    _cycle(3), _cycle(4), _cycle(5), _cycle(6),
    _cycle(4, [0, 1, 0, 1]),
    _pat(4, [(0, 2), (0, 3), (1, 2), (1, 3)], name="bifan"),
    _pat(4, [(0, 1), (0, 2), (0, 3)], name="out_star3"),
    _pat(4, [(0, 1), (1, 0), (0, 2), (2, 0), (0, 3), (3, 0)], name="bistar3"),
    _pat(4, [(a, b) for a in range(4) for b in range(4) if a != b], name="complete4"),
    _pat(5, [(0, 1), (1, 0), (1, 2), (2, 1), (2, 3), (3, 2), (3, 4), (4, 3)], name="bipath5"),
    _pat(4, [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)], name="cycle3_plus_sink"),
    _pat(5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (2, 4)], [0, 1, 0, 1, 2], name="cycle4_hat"),
]


def _random_patterns(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        k = int(rng.integers(2, 7))
        out.append(synth.random_pattern(rng, k, float(rng.uniform(0.2, 0.8)), n_vlab=1 + i % 2,
                                        n_elab=1))
    return out


@pytest.mark.parametrize("sp", SYMMETRIC + _random_patterns(40, 7),
                         ids=lambda p: p.name or f"k{p.k}m{p.mp}")
def test_automorphism_group_is_complete(hm, sp):
    """The group the library breaks is the whole label-preserving group (or 1)."""
    want = _brute_aut(sp)
    got = hm.Pattern.from_synth(sp).automorphisms()
    assert got == (want if sp.k >= 3 and want <= 64 else 1), (sp.name, got, want)


def test_named_groups(hm):
    sizes = {p.name: hm.Pattern.from_synth(p).automorphisms() for p in SYMMETRIC}
    assert sizes["cycle4"] == 4 and sizes["cycle4_0101"] == 2
    assert sizes["bifan"] == 4 and sizes["complete4"] == 24
    assert sizes["out_star3"] == 6 and sizes["bipath5"] == 2
    big = _pat(5, [(a, b) for a in range(5) for b in range(5) if a != b], name="complete5")
    assert hm.Pattern.from_synth(big).automorphisms() == 1   # 120 > 64: searched map by map
    labelled = synth.config2_patterns()
    assert [hm.Pattern.from_synth(p).automorphisms() for p in labelled] == [1, 1, 2]


def _graphs():
    yield "hubs40", synth.small_random_graph(40, 0.25, 1, 1, seed=3, recip=0.5, hub=True)
    yield "complete7", synth.complete_digraph(7)
    g = synth.config2_graph(scale=10)
    yield "rmat10_2lab", synth.Graph(g.n, g.src, g.dst, (g.vlab % 2).astype(np.int32),
                                     np.zeros(g.m, np.int32))


@pytest.mark.gpu
@pytest.mark.parametrize("name,g", list(_graphs()), ids=lambda x: x if isinstance(x, str) else "")
def test_symmetric_patterns_equal_the_oracle(hm, name, g):
    assert torch.cuda.is_available()
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    pats = [p for p in SYMMETRIC if p.k <= (5 if name != "rmat10_2lab" else 4)]
    try:
        for sym in (1, -1):
            hm.set_tuning(symmetry=sym)
            for sp in pats:
                P = hm.Pattern.from_synth(sp)
                for mode in (oracle.MONO, oracle.INDUCED):
                    want_c, want_rows = og.match(sp, mode)
                    assert hm.count_matches(G, P, mode) == want_c, (name, sp.name, mode, sym)
                    rows = hm.enumerate_matches(G, P, mode).cpu().numpy()
                    np.testing.assert_array_equal(rows, want_rows)
            # batched: the same patterns in one launch
            P = [hm.Pattern.from_synth(p) for p in pats]
            counts = hm.count_batch(G, P, hm.INDUCED)
            rows = hm.enumerate_batch(G, P, hm.INDUCED, counts=counts)
            for sp, c, r in zip(pats, counts, rows):
                want_c, want_rows = og.match(sp, oracle.INDUCED)
                assert c == want_c
                np.testing.assert_array_equal(r.cpu().numpy(), want_rows)
    finally:
        hm.set_tuning()
        G.close()
        og.close()


@pytest.mark.gpu
def test_symmetry_with_parts_and_static_count(hm):
    """Arc-range parts still partition the matches; the allocation-free count agrees."""
    g = synth.small_random_graph(60, 0.2, 1, 1, seed=9, recip=0.4, hub=True)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    try:
        for sp in (_cycle(4), SYMMETRIC[5], SYMMETRIC[6]):
            P = hm.Pattern.from_synth(sp)
            for mode in (oracle.MONO, oracle.INDUCED):
                want = og.match(sp, mode, rows=False)[0]
                assert sum(hm.count_matches_part(G, P, mode, i, 3) for i in range(3)) == want
                c = ctypes.c_uint64()
                st = hm.lib.hm_count_matches_static(G.handle, P.handle, int(mode), ctypes.byref(c),
                                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
                assert st == hm.binding.HM_OK and c.value == want
    finally:
        G.close()
        og.close()
