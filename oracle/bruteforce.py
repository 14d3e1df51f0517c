"""Brute-force matcher -- TEST INFRASTRUCTURE ONLY.

Tries every injective map f: V1 -> V2 (itertools.permutations) and keeps
those that satisfy the definition of Sec. II-A: Eq. (2) equal vertex labels,
Eq. (3) every pattern arc maps to a target arc with an equal label, and
Eq. (1) -- "<=>" for induced subgraph isomorphism, "=>" for monomorphism.
Only for tiny inputs (n!/(n-k)! maps).  Shares no code with the C oracle
or with the CUDA library.
"""
from __future__ import annotations

import itertools

import numpy as np


def matches(n, src, dst, vlab, elab, k, psrc, pdst, pvlab, pelab, induced: bool) -> np.ndarray:
    """All matches as an int32 array [count, k], rows (f(0),...,f(k-1)), sorted."""
    tarc = {(int(a), int(b)): int(l) for a, b, l in zip(src, dst, elab)}
    parc = {(int(a), int(b)): int(l) for a, b, l in zip(psrc, pdst, pelab)}
    vl = [int(x) for x in vlab]
    pl = [int(x) for x in pvlab]
    found = []
    for f in itertools.permutations(range(n), k):
        if any(vl[f[i]] != pl[i] for i in range(k)):
            continue
        ok = True
        for a in range(k):
            for b in range(k):
                if a == b:
                    continue
                t = tarc.get((f[a], f[b]))
                if (a, b) in parc:
                    if t is None or t != parc[(a, b)]:
                        ok = False
                        break
                elif induced and t is not None:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            found.append(f)
    out = np.array(sorted(found), dtype=np.int32).reshape(-1, k)
    return out


def matches_of(graph, pattern, induced: bool) -> np.ndarray:
    return matches(graph.n, graph.src, graph.dst, graph.vlab, graph.elab, pattern.k,
                   pattern.src, pattern.dst, pattern.vlab, pattern.elab, induced)
