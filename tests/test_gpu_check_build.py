"""The bounds-checked build (HM_CHECK=1, libhipermotif_check.so).

Every index a kernel forms into a graph array is tested there against the
array's length, and the first one out of range is recorded per graph
(hm_check_status).  On a valid graph none may occur: across graphs with
hubs, reciprocal arcs and labels, patterns of 2..6 vertices in both modes,
every search path (knobs, symmetry breaking, shared position-0 states,
batched launches, the allocation-free count) must leave the record empty
and return the oracle's counts and rows.  The checked library runs in a
child process (the environment variable selects it at import).
"""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import ctypes
import numpy as np
import torch
import oracle, synth
import paper_2507_04130_gb300 as hm

assert hm.lib._name.endswith("libhipermotif_check.so"), hm.lib._name
rng = np.random.default_rng(41)
graphs = [synth.small_random_graph(50, 0.2, 2, 2, seed=3, recip=0.4, hub=True),
          synth.er_graph(400, 6000, 3, 2, seed=4),
          synth.config2_graph(scale=11)]
knobs = [{}, {"arc_filter": -1}, {"leaf_flatten": -1, "pair_mode": 1}, {"lookahead": 1, "warps_per_state": 4},
         {"symmetry": -1, "seeds_per_fetch": 8}]
cases = 0
for g in graphs:
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    pats = [synth.random_pattern(rng, k, float(rng.uniform(0.3, 0.8)), n_vlab=int(g.vlab.max()) + 1,
                                 n_elab=int(g.elab.max()) + 1) for k in (2, 3, 3, 4, 4, 5, 6)]
    pats += synth.config2_patterns()
    for kn in knobs:
        hm.set_tuning(**kn)
        for sp in pats:
            P = hm.Pattern.from_synth(sp)
            for mode in (oracle.MONO, oracle.INDUCED):
                want_c, want_rows = og.match(sp, mode)
                assert hm.count_matches(G, P, mode) == want_c
                np.testing.assert_array_equal(hm.enumerate_matches(G, P, mode).cpu().numpy(), want_rows)
                cases += 1
        hm.set_tuning()
        v = hm.check_status(G)
        assert v == 0, hex(v)
    P = [hm.Pattern.from_synth(sp) for sp in pats]
    counts = hm.count_batch(G, P, hm.INDUCED)
    rows = hm.enumerate_batch(G, P, hm.INDUCED, counts=counts)
    for sp, c, r in zip(pats, counts, rows):
        want_c, want_rows = og.match(sp, oracle.INDUCED)
        assert c == want_c
        np.testing.assert_array_equal(r.cpu().numpy(), want_rows)
    c = ctypes.c_uint64()
    st = hm.lib.hm_count_matches_static(G.handle, P[3].handle, int(hm.MONO), ctypes.byref(c),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == hm.binding.HM_OK and c.value == og.match(pats[3], oracle.MONO, rows=False)[0]
    v = hm.check_status(G)
    assert v == 0, hex(v)
    G.close()
    og.close()
print("clean", cases)
"""


def test_check_build_is_clean_and_exact():
    from paper_2507_04130_gb300 import _build

    _build.build(check=True)
    env = dict(os.environ, HM_CHECK="1")
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", _CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "clean" in r.stdout


def test_default_build_has_no_checks():
    import paper_2507_04130_gb300 as hm
    import synth

    G = hm.Graph.from_synth(synth.small_random_graph(10, 0.3, 1, 1, seed=1))
    try:
        with pytest.raises(hm.HMError) as ei:
            hm.check_status(G)
        assert ei.value.status == hm.binding.HM_ERR_ARG
    finally:
        G.close()
