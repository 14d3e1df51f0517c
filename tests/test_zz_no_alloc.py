"""hm_count_matches_static: counting without any device allocation.

Some callers cannot allocate device memory while they match (their device
memory is carved up in advance by another allocator, or a cudaMalloc that may
synchronise the device is not acceptable in their loop).  This entry point
takes its working memory from a fixed file-scope device array instead.  It
must return exactly what the allocating hm_count_matches returns, on two calls
in a row (the array keeps the previous call's contents between calls), and it
must refuse graphs larger than the array can serve.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2507_04130_gb300 as mod
    assert torch.cuda.is_available()
    return mod


def _static_count(hm, G, P, mode):
    c = ctypes.c_uint64()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = hm.lib.hm_count_matches_static(G.handle, P.handle, int(mode), ctypes.byref(c), stream)
    return st, int(c.value)


def _cases():
    rng = np.random.default_rng(11)
    graphs = [synth.er_graph(400, 6000, 3, 2, seed=7),
              synth.config2_graph(scale=12),
              synth.small_random_graph(30, 0.35, 2, 2, seed=3, recip=0.5, hub=True)]
    pats = [synth.config1_pattern()] + synth.config2_patterns()
    pats.append(synth.Pattern(2, np.array([0], np.int32), np.array([1], np.int32),
                              np.array([0, 1], np.int32), np.array([0], np.int32), "arc"))
    pats += [synth.random_pattern(rng, int(rng.integers(3, 6)), 0.6, n_vlab=2, n_elab=2)
             for _ in range(4)]
    return graphs, pats


def test_static_count_equals_allocating_count_on_consecutive_calls(hm):
    graphs, pats = _cases()
    for g in graphs:
        G = hm.Graph.from_synth(g)
        for sp in pats:
            P = hm.Pattern.from_synth(sp)
            for mode in (hm.MONO, hm.INDUCED):
                want = hm.count_matches(G, P, mode)
                for _ in range(2):
                    st, got = _static_count(hm, G, P, mode)
                    assert st == hm.binding.HM_OK
                    assert got == want, (sp.name, mode, got, want)


def test_static_count_rejects_graphs_beyond_its_array(hm):
    limit = hm.binding.HM_STATIC_MAX_ARCS
    g = synth.er_graph(4000, limit + 1, 2, 2, seed=5)
    G = hm.Graph.from_synth(g)
    P = hm.Pattern.from_synth(synth.config1_pattern())
    st, _ = _static_count(hm, G, P, hm.MONO)
    assert st == hm.binding.HM_ERR_CAPACITY
    # the entry point stays usable on a graph within the limit
    small = synth.er_graph(300, 4000, 3, 1, seed=2)
    Gs = hm.Graph.from_synth(small)
    st, got = _static_count(hm, Gs, P, hm.MONO)
    assert st == hm.binding.HM_OK and got == hm.count_matches(Gs, P, hm.MONO)
