"""The query server: continuous batching over one resident graph.

Each query's result (count and sorted rows) must be the same whether it runs
alone or mixed with others that arrive while earlier batches are on the GPU,
under any memory budget.
"""
from __future__ import annotations

import threading
import time

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


def _queries(seed, count, n_vlab, n_elab):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        k = int(rng.integers(2, 8))
        p = synth.random_pattern(rng, k, float(rng.uniform(0.4, 1.0)), n_vlab=n_vlab, n_elab=n_elab,
                                 name=f"q{i}")
        out.append((p, int(rng.integers(0, 2))))
    return out


def test_each_result_is_the_same_alone_and_in_the_mix(hm):
    g = synth.config2_graph(scale=13)
    G = hm.Graph.from_synth(g)
    qs = _queries(5, 80, 8, 4)
    alone = []
    for p, mode in qs:
        P = hm.Pattern.from_synth(p)
        alone.append((hm.count_matches(G, P, mode), hm.enumerate_matches(G, P, mode).cpu().numpy()))
    srv = hm.Server(G, slots=4, max_batch=16)
    try:
        ids = []

        def client(part):
            for j in range(part, len(qs), 3):
                p, mode = qs[j]
                ids.append((j, srv.submit(p, mode, want_rows=True)))
                time.sleep(0.0005 * (j % 4))

        threads = [threading.Thread(target=client, args=(t,)) for t in range(3)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for j, qid in ids:
            r = srv.result(qid)
            assert r["count"] == alone[j][0]
            assert not r["rows_dropped"]
            got = r["rows"] if r["rows"] is not None else np.zeros((0, qs[j][0].k), np.int32)
            np.testing.assert_array_equal(got, alone[j][1])
            assert r["latency_ms"] > 0
        st = srv.stats()
        assert st["completed"] == len(qs) and st["batches"] >= 1
    finally:
        srv.close()


def test_server_matches_the_oracle_on_a_small_graph(hm):
    g = synth.small_random_graph(40, 0.25, 2, 2, seed=9, recip=0.5, hub=True)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    qs = _queries(6, 30, 2, 2)
    srv = hm.Server(G, slots=2, max_batch=8)
    try:
        ids = [srv.submit(p, mode) for p, mode in qs]
        for (p, mode), qid in zip(qs, ids):
            r = srv.result(qid)
            c, rows = og.match(p, mode)
            assert r["count"] == c and not r["rows_dropped"]
            got = r["rows"] if r["rows"] is not None else np.zeros((0, p.k), np.int32)
            np.testing.assert_array_equal(got, rows)
    finally:
        srv.close()


# what the server charges: 24 B per target arc whose labels fit the query's
# seeding arc (every arc, with one vertex and one arc label), and 12 MiB per batch
BATCH_FIXED = 12 << 20


def test_admission_by_memory_budget_and_dropped_rows(hm):
    g = synth.er_graph(2000, 30000, 1, 1, seed=3)
    G = hm.Graph.from_synth(g)
    per_query = 24 * g.m + BATCH_FIXED
    p = synth.Pattern(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32),
                      np.zeros(3, np.int32), np.zeros(2, np.int32), "path3")
    P = hm.Pattern.from_synth(p)
    want = hm.count_matches(G, P, hm.MONO)
    assert want * 3 * 4 > 4096
    # room for exactly one query and almost no rows: every query runs alone, rows are dropped
    srv = hm.Server(G, slots=3, max_batch=8, mem_budget=per_query + 4096)
    try:
        ids = [srv.submit(p, hm.MONO, want_rows=True) for _ in range(6)]
        for qid in ids:
            r = srv.result(qid)
            assert r["count"] == want and r["rows_dropped"] and r["rows"] is None
        st = srv.stats()
        assert st["max_inflight_batches"] == 1 and st["batches"] == 6 and st["rows_dropped"] == 6
    finally:
        srv.close()
    with pytest.raises(hm.HMError):
        hm.Server(G, slots=1, max_batch=1, mem_budget=BATCH_FIXED - 1)


def test_admission_charges_each_query_by_its_seeding_arc(hm):
    """Queries whose seeding arc fits few target arcs are admitted together under a budget
    that holds only one query whose seeding arc fits every arc."""
    g = synth.er_graph(3000, 40000, 4, 1, seed=5)
    G = hm.Graph.from_synth(g)
    few = synth.Pattern(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32),
                        np.array([0, 1, 2], np.int32), np.zeros(2, np.int32), "labelled_path3")
    # a flat charge of 24 B x m + 8 MiB per query would admit two of them per batch
    srv = hm.Server(G, slots=1, max_batch=8, mem_budget=BATCH_FIXED + 24 * g.m // 2 + (8 << 20))
    try:
        ids = [srv.submit(few, hm.MONO, want_rows=True) for _ in range(8)]
        want = hm.count_matches(G, hm.Pattern.from_synth(few), hm.MONO)
        for qid in ids:
            r = srv.result(qid)
            assert r["count"] == want and not r["rows_dropped"]
        assert srv.stats()["batches"] <= 3   # each needs ~1/16 of the arcs: they share batches
    finally:
        srv.close()


def test_batches_overlap_on_the_device(hm):
    g = synth.config2_graph(scale=15)
    G = hm.Graph.from_synth(g)
    qs = _queries(8, 120, 8, 4)
    srv = hm.Server(G, slots=4, max_batch=4)
    try:
        ids = [srv.submit(p, mode, want_rows=False) for p, mode in qs]
        for qid in ids:
            srv.result(qid)
        st = srv.stats()
        assert st["completed"] == len(qs)
        assert st["max_inflight_batches"] >= 2
    finally:
        srv.close()


def test_close_drains_queries_still_waiting_for_memory(hm):
    g = synth.er_graph(2000, 30000, 1, 1, seed=4)
    G = hm.Graph.from_synth(g)
    per_query = 24 * g.m + BATCH_FIXED
    p = synth.Pattern(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32),
                      np.zeros(3, np.int32), np.zeros(2, np.int32), "path3")
    # three slots but memory for one query: most queries wait for memory when close() is called
    srv = hm.Server(G, slots=3, max_batch=8, mem_budget=per_query)
    for _ in range(12):
        srv.submit(p, hm.MONO, want_rows=False)
    t0 = time.perf_counter()
    closer = threading.Thread(target=srv.close)
    closer.start()
    closer.join(120)
    assert not closer.is_alive()
    assert time.perf_counter() - t0 < 120
