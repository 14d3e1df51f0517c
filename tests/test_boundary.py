"""Host-side tests of the C ABI that need no GPU.

  * the library loads and exports every function include/hipermotif.h declares;
  * hm_load_pattern validates patterns and runs Alg. 1 exactly like the
    oracle's plain restatement (hand-worked cases and random patterns);
  * loading a graph without a device fails with a status, not a crash;
  * the Python front end rejects arrays of the wrong length and unusable row
    buffers before it calls the library (the CUDA-tensor cases are marked gpu).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest
import torch

import synth
from oracle import steps
from tests import _golden

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2507_04130_gb300 as mod
    return mod


def _declared():
    text = open(os.path.join(ROOT, "include", "hipermotif.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hm_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(hm):
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(hm.lib, name), name
    assert sorted(hm.binding.EXPORTED) == declared


def test_status_strings(hm):
    for s in range(10):
        assert hm.lib.hm_status_str(s)
    assert hm.lib.hm_status_str(hm.binding.HM_ERR_CAPACITY).decode() == "output capacity too small"


@pytest.mark.parametrize("case", _golden.reorder_cases(), ids=lambda c: c["name"])
def test_pattern_order_hand_worked(hm, case):
    src = [a for a, _ in case["arcs"]]
    dst = [b for _, b in case["arcs"]]
    p = hm.Pattern(case["k"], src, dst, [0] * case["k"], [0] * len(src))
    assert p.order == case["order"]


@pytest.mark.parametrize("seed", range(40))
def test_pattern_order_equals_plain_alg1(hm, seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 21))
    p = synth.random_pattern(rng, k, float(rng.uniform(0.05, 0.8)), n_vlab=2, n_elab=2)
    assert hm.Pattern.from_synth(p).order == steps.structural_reorder(k, p.src, p.dst)


def test_config_patterns_order(hm):
    for p in synth.config2_patterns() + synth.config3_patterns() + synth.config4_patterns(count=32):
        assert hm.Pattern.from_synth(p).order == steps.structural_reorder(p.k, p.src, p.dst)


@pytest.mark.parametrize("k,src,dst,status", [
    (1, [0], [0], "HM_ERR_PATTERN"),                       # k < 2
    (21, [0], [1], "HM_ERR_PATTERN"),                      # k > 20
    (3, [], [], "HM_ERR_PATTERN"),                         # no arc
    (3, [0, 1], [0, 2], "HM_ERR_SELF_LOOP"),
    (3, [0, 0], [1, 1], "HM_ERR_DUP_EDGE"),
    (4, [0, 2], [1, 3], "HM_ERR_PATTERN"),                 # not weakly connected
    (3, [0, 1], [1, 5], "HM_ERR_ARG"),                     # id out of range
])
def test_pattern_validation(hm, k, src, dst, status):
    with pytest.raises(hm.HMError) as ei:
        hm.Pattern(k, src, dst, [0] * max(k, 1), [0] * len(src))
    assert ei.value.status == getattr(hm.binding, status)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_graph_load_without_device_reports_status(hm):
    arrs = [np.array(a, np.int32) for a in ([0, 1], [1, 2], [0, 0, 0], [0, 0])]
    h = ctypes.c_void_p()
    st = hm.lib.hm_load_graph(3, 2, *[ctypes.c_void_p(a.ctypes.data) for a in arrs], 0, None,
                              ctypes.byref(h))
    assert st in (hm.binding.HM_ERR_NO_DEVICE, hm.binding.HM_ERR_CUDA)


def test_graph_load_rejects_bad_arguments_before_the_device(hm):
    h = ctypes.c_void_p()
    assert hm.lib.hm_load_graph(-1, 0, None, None, None, None, 0, None, ctypes.byref(h)) == \
        hm.binding.HM_ERR_ARG
    assert hm.lib.hm_load_graph(3, 2, None, None, None, None, 0, None, ctypes.byref(h)) == \
        hm.binding.HM_ERR_ARG


@pytest.mark.parametrize("bad", [dict(extend_min_blocks=7), dict(split_min=1), dict(pair_mode=2),
                                 dict(seeds_per_fetch=5000), dict(poll_every=3),
                                 dict(poll_every=1 << 17), dict(leaf_flatten=2), dict(arc_filter=-2),
                                 dict(share_seeds=2), dict(symmetry=2), dict(symmetry=-2),
                                 dict(warps_per_state=3), dict(warps_per_state=8), dict(warps_per_state=-1),
                                 dict(lookahead=2), dict(lookahead=-2)])
def test_tuning_rejects_bad_values(hm, bad):
    before = hm.get_tuning()
    with pytest.raises(hm.HMError) as ei:
        hm.set_tuning(**bad)
    assert ei.value.status == hm.binding.HM_ERR_ARG
    assert hm.get_tuning() == before


def test_tuning_defaults_roundtrip(hm):
    hm.set_tuning(extend_min_blocks=6, split_min=128, pair_mode=1, seeds_per_fetch=4, poll_every=8)
    assert hm.get_tuning() == dict(extend_min_blocks=6, split_min=128, pair_mode=1, seeds_per_fetch=4,
                                   poll_every=8, leaf_flatten=1, arc_filter=1, share_seeds=1, symmetry=1,
                                   warps_per_state=0, lookahead=-1)
    hm.set_tuning(leaf_flatten=-1, arc_filter=-1, symmetry=-1)
    assert hm.get_tuning()["leaf_flatten"] == -1 and hm.get_tuning()["arc_filter"] == -1
    assert hm.get_tuning()["symmetry"] == -1
    hm.set_tuning()
    assert hm.get_tuning() == dict(extend_min_blocks=4, split_min=64, pair_mode=0, seeds_per_fetch=1,
                                   poll_every=128, leaf_flatten=1, arc_filter=1, share_seeds=1, symmetry=1,
                                   warps_per_state=0, lookahead=-1)


def _bfs_order(k, src, dst):
    adj = {v: set() for v in range(k)}
    for a, b in zip(src, dst):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    order, seen = [0], {0}
    for v in order:
        for w in sorted(adj[v]):
            if w not in seen:
                seen.add(w)
                order.append(w)
    return order


def test_pattern_with_a_given_order(hm):
    rng = np.random.default_rng(3)
    for _ in range(20):
        k = int(rng.integers(2, 12))
        p = synth.random_pattern(rng, k, 0.4, n_vlab=2, n_elab=2)
        order = _bfs_order(k, p.src, p.dst)
        assert hm.Pattern.from_synth(p, order=order).order == order
    p = synth.Pattern(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32),
                      np.zeros(3, np.int32), np.zeros(2, np.int32))
    with pytest.raises(hm.HMError) as ei:                       # position 1 unanchored
        hm.Pattern.from_synth(p, order=[0, 2, 1])
    assert ei.value.status == hm.binding.HM_ERR_PATTERN
    with pytest.raises(hm.HMError) as ei:                       # not a permutation
        hm.Pattern.from_synth(p, order=[0, 1, 1])
    assert ei.value.status == hm.binding.HM_ERR_ARG


def test_pattern_arrays_must_have_the_declared_lengths(hm):
    with pytest.raises(ValueError, match="vlab"):
        hm.Pattern(3, [0, 1], [1, 2], [0, 0], [0, 0])          # vlab short of k
    with pytest.raises(ValueError, match="dst"):
        hm.Pattern(3, [0, 1], [1], [0, 0, 0], [0, 0])
    with pytest.raises(ValueError, match="elab"):
        hm.Pattern(3, [0, 1], [1, 2], [0, 0, 0], [0])


class _FakeGraph:
    handle = None
    n = 8


def test_row_buffers_are_checked_before_the_call(hm):
    P = hm.Pattern(3, [0, 1], [1, 2], [0, 0, 0], [0, 0])
    G = _FakeGraph()
    host = torch.empty(30, dtype=torch.int32)
    with pytest.raises(ValueError, match="CUDA"):
        hm.enumerate_matches(G, P, hm.MONO, out=host)
    with pytest.raises(ValueError, match="CUDA"):
        hm.enumerate_matches_part(G, P, hm.MONO, 0, 1, host)
    with pytest.raises(ValueError, match="capacity"):
        hm.enumerate_matches(G, P, hm.MONO, capacity=-1)


@pytest.mark.gpu
def test_device_row_buffers_and_masks_are_checked_before_the_call(hm):
    P = hm.Pattern(3, [0, 1], [1, 2], [0, 0, 0], [0, 0])
    G = _FakeGraph()                    # never reaches the library
    dev = torch.empty(30, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError, match="exceeds"):
        hm.enumerate_matches(G, P, hm.MONO, out=dev, capacity=11)   # 30 int32 hold 10 rows
    with pytest.raises(ValueError, match="int32"):
        hm.enumerate_matches(G, P, hm.MONO, out=dev.to(torch.int64))
    with pytest.raises(ValueError, match="contiguous"):
        hm.enumerate_matches(G, P, hm.MONO, out=dev.view(10, 3).t())
    with pytest.raises(ValueError, match="mask"):
        hm.count_matches_rooted(G, P, hm.MONO, 0, np.ones(G.n - 1, np.uint8))
