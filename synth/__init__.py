"""Seeded synthetic inputs for labelled directed subgraph matching.

Target graphs and pattern graphs shaped like the workloads of Sec. IV-A
(Erdos-Renyi graphs with uniform random labels, power-law graphs, and
connectome-like property graphs with cell-type vertex labels and synapse-type
edge labels), plus Poisson query arrivals for the serving workload.

This module holds no matching arithmetic.  It only draws arrays; the CUDA path
and the CPU oracle both take these arrays as plain inputs, so neither depends
on the other through it.  Every generator takes an explicit seed and draws
from numpy's PCG64, so its output is a pure function of its arguments.

Conventions shared by every generator:
  * a target graph is a simple digraph: no self-loops, no duplicate (u, v);
  * vertex ids are int32 in [0, n); labels are int32 >= 0;
  * arcs are given as two int32 arrays ``src``, ``dst`` of equal length m.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Graph", "Pattern", "er_graph", "rmat_graph", "chung_lu_graph",
    "small_random_graph", "complete_digraph", "random_pattern",
    "zipf_weights", "CELL_TYPE_WEIGHTS", "config1_graph", "config1_pattern",
    "config2_graph", "config2_patterns", "config3_graph", "config3_patterns",
    "config4_patterns", "config5_arrivals", "cached",
]


@dataclass(frozen=True)
class Graph:
    n: int
    src: np.ndarray   # int32[m]
    dst: np.ndarray   # int32[m]
    vlab: np.ndarray  # int32[n]
    elab: np.ndarray  # int32[m]

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


@dataclass(frozen=True)
class Pattern:
    k: int
    src: np.ndarray   # int32[mp]
    dst: np.ndarray   # int32[mp]
    vlab: np.ndarray  # int32[k]
    elab: np.ndarray  # int32[mp]
    name: str = ""

    @property
    def mp(self) -> int:
        return int(self.src.shape[0])


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# label distributions
# ---------------------------------------------------------------------------

def zipf_weights(s: float, count: int) -> np.ndarray:
    """Probabilities proportional to (i+1)^-s for i in [0, count)."""
    w = np.arange(1, count + 1, dtype=np.float64) ** (-s)
    return w / w.sum()


#: cell-type frequencies of the connectome-shaped workload (6 types)
CELL_TYPE_WEIGHTS = np.array([0.40, 0.25, 0.15, 0.10, 0.06, 0.04])


def _labels(rng, count, weights=None, n_values=None) -> np.ndarray:
    if weights is not None:
        return _i32(rng.choice(len(weights), size=count, p=np.asarray(weights) / np.sum(weights)))
    return _i32(rng.integers(0, n_values, size=count))


# ---------------------------------------------------------------------------
# arc-set helpers
# ---------------------------------------------------------------------------

def _sorted_unique(keys: np.ndarray) -> np.ndarray:
    """Distinct keys, ascending (sort-based; avoids numpy's slow hash path)."""
    keys = np.sort(keys, kind="stable")
    if keys.shape[0] == 0:
        return keys
    keep = np.empty(keys.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(keys[1:], keys[:-1], out=keep[1:])
    return keys[keep]


def _first_unique(keys: np.ndarray, limit: int | None = None) -> np.ndarray:
    """Distinct keys in order of first appearance (optionally the first `limit`)."""
    order = np.argsort(keys, kind="stable")
    sk = keys[order]
    first = np.empty(sk.shape[0], dtype=bool)
    if sk.shape[0]:
        first[0] = True
        np.not_equal(sk[1:], sk[:-1], out=first[1:])
    idx = np.sort(order[first])
    if limit is not None:
        idx = idx[:limit]
    return keys[idx]


# ---------------------------------------------------------------------------
# target graphs
# ---------------------------------------------------------------------------

def er_graph(n: int, m: int, n_vlab: int, n_elab: int, seed: int) -> Graph:
    """Directed G(n, m): m distinct ordered pairs (i, j), i != j, uniformly at random.

    Pairs are drawn i.i.d. uniform over the n(n-1) ordered non-loop pairs and
    the first m distinct ones are kept, which is a uniform m-subset.
    Vertex labels uniform over [0, n_vlab), edge labels uniform over [0, n_elab).
    """
    if m > n * (n - 1):
        raise ValueError("m exceeds n(n-1)")
    rng = _rng(seed)
    keys = np.empty(0, dtype=np.int64)
    while keys.shape[0] < m:
        b = max(2 * (m - keys.shape[0]), 1024)
        u = rng.integers(0, n, size=b, dtype=np.int64)
        v = rng.integers(0, n - 1, size=b, dtype=np.int64)
        v = v + (v >= u)                      # uniform over [0,n) \ {u}
        keys = _first_unique(np.concatenate([keys, u * n + v]))
    keys = keys[:m]
    src, dst = keys // n, keys % n
    vlab = _labels(rng, n, n_values=n_vlab)
    elab = _labels(rng, m, n_values=n_elab)
    return Graph(n, _i32(src), _i32(dst), vlab, elab)


def rmat_graph(scale: int, n_samples: int, a: float, b: float, c: float, seed: int,
               vlab_weights, n_elab: int) -> Graph:
    """Directed R-MAT graph (Chakrabarti et al.), Graph500-style cleanup.

    Each of `n_samples` arcs picks one quadrant per level with probabilities
    (a, b, c, d = 1-a-b-c); the first bit is the source's, the second the
    destination's, most significant level first.  Self-loops and duplicate
    (u, v) are removed, then vertex ids are relabelled by a seeded random
    permutation so ids carry no locality.
    """
    n = 1 << scale
    rng = _rng(seed)
    src = np.zeros(n_samples, dtype=np.int64)
    dst = np.zeros(n_samples, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for _ in range(scale):
        r = rng.random(n_samples)
        sbit = r >= ab
        dbit = ((r >= a) & (r < ab)) | (r >= abc)
        src = (src << 1) | sbit
        dst = (dst << 1) | dbit
    keep = src != dst
    keys = _sorted_unique(src[keep] * n + dst[keep])
    src, dst = keys // n, keys % n
    perm = rng.permutation(n).astype(np.int64)
    src, dst = perm[src], perm[dst]
    vlab = _labels(rng, n, weights=vlab_weights)
    elab = _labels(rng, src.shape[0], n_values=n_elab)
    return Graph(n, _i32(src), _i32(dst), vlab, elab)


def _discrete_power_law(rng, count, exponent, dmin, dmax) -> np.ndarray:
    support = np.arange(dmin, dmax + 1, dtype=np.float64)
    pmf = support ** (-exponent)
    pmf /= pmf.sum()
    return support[rng.choice(support.shape[0], size=count, p=pmf)]


def _alias_table(weights: np.ndarray):
    """Walker's alias method (Vose's construction): O(1) draws proportional to `weights`."""
    n = weights.shape[0]
    scaled = weights.astype(np.float64) * (n / weights.sum())
    prob = np.ones(n, dtype=np.float64)
    alias = np.arange(n, dtype=np.int64)
    small = np.nonzero(scaled < 1.0)[0].tolist()
    large = np.nonzero(scaled >= 1.0)[0].tolist()
    sc = scaled.tolist()
    while small and large:
        s_, l_ = small.pop(), large.pop()
        prob[s_] = sc[s_]
        alias[s_] = l_
        sc[l_] = sc[l_] + sc[s_] - 1.0
        (small if sc[l_] < 1.0 else large).append(l_)
    return prob, alias


def _alias_draw(rng, table, count: int) -> np.ndarray:
    prob, alias = table
    i = rng.integers(0, prob.shape[0], size=count, dtype=np.int64)
    return np.where(rng.random(count) < prob[i], i, alias[i])


def _merge_unique(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Distinct keys of two ascending arrays, ascending (one stable run-merging sort)."""
    keys = np.concatenate([a, b])
    keys.sort(kind="stable")
    if keys.shape[0] == 0:
        return keys
    keep = np.empty(keys.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(keys[1:], keys[:-1], out=keep[1:])
    return keys[keep]


def chung_lu_graph(n: int, exponent: float, dmin: int, dmax: int, n_unique: int,
                   n_recip: int, vlab_weights, n_elab: int, seed: int) -> Graph:
    """Directed Chung-Lu graph with power-law in- and out-weights and added reciprocity.

    Out- and in-weights are drawn independently from a discrete power law
    proportional to d^-exponent on [dmin, dmax].  Arcs are drawn (alias tables)
    with source proportional to the out-weight and destination proportional to
    the in-weight, self-loops dropped, until at least `n_unique` distinct arcs
    exist; a seeded uniform subset of exactly `n_unique` of them is kept.  Then
    `n_recip` of those arcs are chosen uniformly and their reverses added
    (reverses already present are not duplicated).
    """
    rng = _rng(seed)
    w_out = _discrete_power_law(rng, n, exponent, dmin, dmax)
    w_in = _discrete_power_law(rng, n, exponent, dmin, dmax)
    t_out, t_in = _alias_table(w_out), _alias_table(w_in)
    keys = np.empty(0, dtype=np.int64)
    chunk = 1 << 24
    while keys.shape[0] < n_unique:
        want = int(1.1 * (n_unique - keys.shape[0])) + 1024
        parts = []
        for lo in range(0, want, chunk):
            b = min(chunk, want - lo)
            u = _alias_draw(rng, t_out, b)
            v = _alias_draw(rng, t_in, b)
            k = u[u != v] * n + v[u != v]
            k.sort()
            parts.append(k)
        new = np.concatenate(parts)
        new.sort(kind="stable")
        keys = _merge_unique(keys, new)
    excess = keys.shape[0] - n_unique
    if excess > 0:
        keep = np.ones(keys.shape[0], dtype=bool)
        keep[rng.choice(keys.shape[0], size=excess, replace=False)] = False
        keys = keys[keep]
    pick = rng.choice(keys.shape[0], size=n_recip, replace=False)
    rev = (keys[pick] % n) * n + keys[pick] // n
    rev.sort()
    keys = _merge_unique(keys, rev)
    src, dst = keys // n, keys % n
    vlab = _labels(rng, n, weights=vlab_weights)
    elab = _labels(rng, keys.shape[0], n_values=n_elab)
    return Graph(n, _i32(src), _i32(dst), vlab, elab)


def small_random_graph(n: int, p: float, n_vlab: int, n_elab: int, seed: int,
                       recip: float = 0.0, hub: bool = False) -> Graph:
    """Small digraph for exhaustive tests: each ordered pair i != j is an arc with prob. p.

    `recip` adds the reverse of each arc with that probability; `hub` makes
    vertex 0 adjacent to every other vertex in both directions.
    """
    rng = _rng(seed)
    A = rng.random((n, n)) < p
    np.fill_diagonal(A, False)
    if recip > 0:
        R = rng.random((n, n)) < recip
        A = A | (A.T & R)
    if hub and n > 1:
        A[0, 1:] = True
        A[1:, 0] = True
    np.fill_diagonal(A, False)
    src, dst = np.nonzero(A)
    vlab = _labels(rng, n, n_values=n_vlab)
    elab = _labels(rng, src.shape[0], n_values=n_elab)
    return Graph(n, _i32(src), _i32(dst), vlab, elab)


def complete_digraph(n: int) -> Graph:
    """All n(n-1) ordered pairs, one vertex label and one edge label (both 0)."""
    A = ~np.eye(n, dtype=bool)
    src, dst = np.nonzero(A)
    return Graph(n, _i32(src), _i32(dst), np.zeros(n, np.int32), np.zeros(src.shape[0], np.int32))


# ---------------------------------------------------------------------------
# pattern graphs
# ---------------------------------------------------------------------------

def _weakly_connected(k: int, src, dst) -> bool:
    parent = list(range(k))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in zip(src, dst):
        parent[find(int(a))] = find(int(b))
    return len({find(i) for i in range(k)}) == 1


def random_pattern(rng: np.random.Generator, k: int, density: float, *, vlab_weights=None,
                   n_vlab: int | None = None, n_elab: int = 1, name: str = "") -> Pattern:
    """Random weakly connected pattern: round(density * k(k-1)) distinct arcs, no loops.

    Resamples the arc set until the pattern is weakly connected.
    """
    pairs = [(i, j) for i in range(k) for j in range(k) if i != j]
    n_arcs = int(round(density * len(pairs)))
    n_arcs = min(max(n_arcs, k - 1), len(pairs))
    while True:
        sel = rng.choice(len(pairs), size=n_arcs, replace=False)
        sel.sort()
        src = [pairs[s][0] for s in sel]
        dst = [pairs[s][1] for s in sel]
        if _weakly_connected(k, src, dst):
            break
    vlab = _labels(rng, k, weights=vlab_weights, n_values=n_vlab)
    elab = _labels(rng, n_arcs, n_values=n_elab)
    return Pattern(k, _i32(src), _i32(dst), vlab, elab, name)


def _pattern(k, arcs, vlab, elab, name) -> Pattern:
    src = [a for a, _ in arcs]
    dst = [b for _, b in arcs]
    return Pattern(k, _i32(src), _i32(dst), _i32(vlab), _i32(elab), name)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

def config1_graph() -> Graph:
    """ER: n=1,000, m=5,000, seed 0, vertex labels U{0..3}, edge labels U{0..2}."""
    return er_graph(1000, 5000, 4, 3, seed=0)


def config1_pattern() -> Pattern:
    """Directed 3-cycle 0->1->2->0, vertex labels (0,1,2), edge labels 0."""
    return _pattern(3, [(0, 1), (1, 2), (2, 0)], [0, 1, 2], [0, 0, 0], "cycle3")


RMAT_ABC = (0.57, 0.19, 0.19)


def config2_graph(scale: int = 20, n_samples: int | None = None, seed: int = 1) -> Graph:
    """R-MAT scale 20, 2^24 samples, (a,b,c,d)=(.57,.19,.19,.05), seed 1.

    Vertex labels Zipf(s=1.2) over 8 values, edge labels uniform over 4 values.
    Smaller `scale` gives the same recipe at a reduced size (16 samples per vertex).
    """
    if n_samples is None:
        n_samples = 16 << scale
    return rmat_graph(scale, n_samples, *RMAT_ABC, seed=seed,
                      vlab_weights=zipf_weights(1.2, 8), n_elab=4)


def config2_patterns() -> list[Pattern]:
    """Feed-forward loop plus one out-edge, bi-fan, 4-cycle; vertex labels (0,1,0,1), edge labels 0."""
    lab = [0, 1, 0, 1]
    return [
        _pattern(4, [(0, 1), (1, 2), (0, 2), (2, 3)], lab, [0] * 4, "ffl_out"),
        _pattern(4, [(0, 2), (0, 3), (1, 2), (1, 3)], lab, [0] * 4, "bifan"),
        _pattern(4, [(0, 1), (1, 2), (2, 3), (3, 0)], lab, [0] * 4, "cycle4"),
    ]


def config3_graph(n: int = 300_000, n_unique: int = 142_500_000, n_recip: int = 7_500_000,
                  seed: int = 3) -> Graph:
    """Connectome-shaped: Chung-Lu, exponent 2.1, weights in [98, 50000], ~150M arcs.

    ~10% of arcs are in reciprocal pairs; vertex labels over 6 cell types
    (0.40/0.25/0.15/0.10/0.06/0.04), edge labels over 3 synapse types.
    Smaller arguments give the same recipe at reduced size.
    """
    dmax = min(50_000, max(n // 6, 200))
    dmin = min(98, max(dmax // 20, 2))
    return chung_lu_graph(n, 2.1, dmin, dmax, n_unique, n_recip, CELL_TYPE_WEIGHTS, 3, seed)


def config3_patterns(seed: int = 3, count: int = 5) -> list[Pattern]:
    """Five 5-vertex patterns, density U[0.5, 0.8] of the 20 ordered pairs, weakly connected."""
    rng = _rng(seed)
    out = []
    for i in range(count):
        d = rng.uniform(0.5, 0.8)
        out.append(random_pattern(rng, 5, d, vlab_weights=CELL_TYPE_WEIGHTS, n_elab=3,
                                  name=f"conn5_{i}"))
    return out


def config4_patterns(seed: int = 2, count: int = 256) -> list[Pattern]:
    """256 patterns, k ~ U{3..6}, density U[0.4, 1.0], vertex labels U{0..7}, edge labels U{0..3}."""
    rng = _rng(seed)
    out = []
    for i in range(count):
        k = int(rng.integers(3, 7))
        d = rng.uniform(0.4, 1.0)
        out.append(random_pattern(rng, k, d, n_vlab=8, n_elab=4, name=f"batch_{i}"))
    return out


def config5_arrivals(rate: float, count: int, seed: int = 4, n_vlab: int = 6, n_elab: int = 3):
    """Open-loop Poisson arrivals of motif queries.

    Returns a list of (arrival_time_s, Pattern, mode) with mode 0 = monomorphism,
    1 = induced; k ~ U{3..7}, density U[0.4, 1.0], labels uniform over the
    target's label sets.
    """
    rng = _rng(seed + int(rate * 1000))
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        k = int(rng.integers(3, 8))
        d = rng.uniform(0.4, 1.0)
        p = random_pattern(rng, k, d, n_vlab=n_vlab, n_elab=n_elab, name=f"q{i}")
        mode = int(rng.integers(0, 2))
        out.append((t, p, mode))
    return out


# ---------------------------------------------------------------------------
# on-disk cache for the large graphs (pure function of the arguments)
# ---------------------------------------------------------------------------

#: bumped whenever a generator's output changes, so stale cache files are not reused
_GENERATOR_VERSION = 2


def cached(name: str, fn, *args, **kwargs) -> Graph:
    """Return fn(*args, **kwargs), memoised as an .npz under $HM_CACHE (default: the user's
    cache directory, $XDG_CACHE_HOME or ~/.cache, subfolder hipermotif_synth)."""
    root = os.environ.get("HM_CACHE") or os.path.join(
        os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache"),
        "hipermotif_synth")
    os.makedirs(root, exist_ok=True)
    key = f"{name}_v{_GENERATOR_VERSION}_" + "_".join(str(a) for a in args) + "_" + "_".join(
        f"{k}{v}" for k, v in sorted(kwargs.items()))
    path = os.path.join(root, key + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        return Graph(int(z["n"]), z["src"], z["dst"], z["vlab"], z["elab"])
    g = fn(*args, **kwargs)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, n=np.int64(g.n), src=g.src, dst=g.dst, vlab=g.vlab, elab=g.elab)
    os.replace(tmp, path)
    return g
