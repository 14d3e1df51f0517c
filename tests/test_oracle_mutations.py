"""The oracle's pins catch plausible mistakes: each test plants one in a copy of oracle.c.

Every mutant is compiled on the CPU into a temporary library and run through a
quick subset of the pins (brute force, complete-digraph closed forms, the
labelled 3-cycle trace identity, the mono/induced completion sum).  The
unmutated source must pass the same subset; each mutant must fail it.
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import bruteforce

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTATIONS = {
    "drop_vertex_label": ("if (g->vlab[c] != P->vlab[p]) return 0;", ""),
    "drop_injectivity": ("if (w->f[P->order[i]] == c) return 0;", ""),
    "drop_edge_label": ("if (!present || lab != P->alab[q][p]) return 0;",
                        "if (!present) return 0;"),
    "drop_induced_nonarc": ("} else if (w->induced && present) {\n      return 0;                                           /* Eq. (1), \"<=\" */",
                            "} else if (0) {\n      return 0;"),
    "swap_domain_direction": ("if (P->from_parent[p]) {", "if (!P->from_parent[p]) {"),
    "transposed_arc_operands": ("present = target_arc(g, c, w->f[q], &lab);",
                                "present = target_arc(g, w->f[q], c, &lab);"),
    "rows_in_visit_order": ("memcpy(w->rows.data + w->rows.len * (size_t)k, w->f, (size_t)k * sizeof(int32_t));",
                            "for (int i_ = 0; i_ < k; ++i_) w->rows.data[w->rows.len * (size_t)k + i_] = w->f[w->P->order[i_]];"),
    "emit_one_level_early": ("if (d == P->k) return emit(w);", "if (d == P->k - 1) return emit(w);"),
    "search_drops_right_half": ("if (x < b) lo = mid + 1; else hi = mid;",
                                "if (x < b) hi = mid; else lo = mid + 1;"),
}


def _pins_pass(lib) -> bool:
    rng = np.random.default_rng(42)
    # brute force, both modes
    for seed in range(6):
        g = synth.small_random_graph(6, 0.5, 2, 2, seed=seed, recip=0.5, hub=seed == 0)
        og = oracle.OracleGraph.from_synth(g, lib=lib)
        for _ in range(3):
            k = int(rng.integers(2, 5))
            p = synth.random_pattern(rng, k, 0.5, n_vlab=2, n_elab=2)
            for mode in (0, 1):
                want = bruteforce.matches_of(g, p, bool(mode))
                cnt, rows = og.match(p, mode, threads=2)
                if cnt != want.shape[0] or not np.array_equal(rows, want):
                    return False
    # complete digraph closed form
    g = synth.complete_digraph(6)
    og = oracle.OracleGraph.from_synth(g, lib=lib)
    p = synth.random_pattern(rng, 3, 0.4, n_vlab=1, n_elab=1)
    if og.match(p, 0, rows=False)[0] != math.perm(6, 3):
        return False
    # labelled 3-cycle trace identity
    g = synth.er_graph(120, 2500, 3, 2, seed=3)
    A0 = np.zeros((g.n, g.n), np.int64)
    sel = g.elab == 0
    A0[g.src[sel], g.dst[sel]] = 1
    D = [np.diag((g.vlab == i).astype(np.int64)) for i in range(3)]
    want = int(np.trace(D[0] @ A0 @ D[1] @ A0 @ D[2] @ A0))
    got = oracle.OracleGraph.from_synth(g, lib=lib).match(synth.config1_pattern(), 0, rows=False)[0]
    if got != want:
        return False
    # mono = sum over induced completions
    g = synth.er_graph(25, 250, 2, 2, seed=8)
    og = oracle.OracleGraph.from_synth(g, lib=lib)
    p = synth.Pattern(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32),
                      np.array([0, 1, 0], np.int32), np.array([0, 1], np.int32))
    holes = [(a, b) for a in range(3) for b in range(3) if a != b and (a, b) not in {(0, 1), (1, 2)}]
    total = 0
    for choice in itertools.product(range(3), repeat=len(holes)):
        src, dst, lab = [0, 1], [1, 2], [0, 1]
        for (a, b), c in zip(holes, choice):
            if c:
                src.append(a); dst.append(b); lab.append(c - 1)
        q = synth.Pattern(3, np.array(src, np.int32), np.array(dst, np.int32), p.vlab,
                          np.array(lab, np.int32))
        total += og.match(q, 1, rows=False)[0]
    return og.match(p, 0, rows=False)[0] == total


def _compile(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    return oracle.load(oracle.build(str(src), str(tmp_path / f"lib{name}.so")))


def test_unmutated_oracle_passes_pin_subset(tmp_path):
    with open(SRC) as f:
        text = f.read()
    assert _pins_pass(_compile(tmp_path, "clean", text))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = text.replace(old, new, 1)
    assert not _pins_pass(_compile(tmp_path, name, mutated))
