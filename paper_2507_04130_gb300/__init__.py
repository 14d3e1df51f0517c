"""GB300-native labelled subgraph matching with the HiPerMotif method.

Python front end of libhipermotif.so (include/hipermotif.h).  It converts
numpy arrays / torch tensors to plain pointers and CUDA streams and calls the
C ABI; PyTorch supplies device memory and streams only.  The library finds
every match of a small pattern in a large target digraph (Sec. II-A) by
reordering the pattern (Alg. 1), validating every target arc as the image of
the pattern's first arc (Alg. 2, Alg. 3), injecting survivors as depth-2
states and extending them in parallel (Sec. III-C).

    g = Graph(n, src, dst, vlab, elab)          # device-resident target
    p = Pattern(k, psrc, pdst, pvlab, pelab)    # runs Alg. 1
    count_matches(g, p, MONO)                   # -> int
    enumerate_matches(g, p, INDUCED)            # -> torch.int32 [count, k] (cuda)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding
from .binding import HM_INDUCED as INDUCED
from .binding import HM_MONO as MONO
from .binding import HMError, check, lib

__all__ = ["Graph", "Pattern", "count_matches", "enumerate_matches", "count_matches_rooted",
           "count_matches_part", "enumerate_matches_part", "count_batch", "enumerate_batch", "autotune", "Server",
           "injected_states", "set_budget", "set_timing", "set_counters", "set_tuning", "get_tuning",
           "last_stats", "check_status", "MONO", "INDUCED",
           "HMError", "binding"]


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _host_i32(a) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a) -> ctypes.c_void_p:
    if isinstance(a, torch.Tensor):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _check_lengths(what: str, arrays, sizes):
    """The library reads exactly these many elements from each array."""
    for name, a, want in zip(("src", "dst", "vlab", "elab"), arrays, sizes):
        if int(a.shape[0]) != int(want):
            raise ValueError(f"{what}: {name} has {int(a.shape[0])} entries, expected {int(want)}")


def _rows_capacity(out: torch.Tensor, k: int, capacity) -> int:
    """Rows that `out` can take; the library writes up to capacity * k int32 there on the device."""
    if not isinstance(out, torch.Tensor) or not out.is_cuda:
        raise ValueError("out must be a CUDA tensor")
    if out.dtype != torch.int32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous int32 tensor")
    have = int(out.numel() // k)
    if capacity is None:
        return have
    if not 0 <= int(capacity) <= have:
        raise ValueError(f"capacity {int(capacity)} exceeds the {have} rows that out holds")
    return int(capacity)


class Graph:
    """A target graph resident in device memory (CSR + CSC + labels), built on the GPU.

    Arrays may be numpy arrays / CPU tensors (copied from the host) or int32
    CUDA tensors (read on the device).
    """

    def __init__(self, n: int, src, dst, vlab, elab, stream=None):
        arrays = [src, dst, vlab, elab]
        on_dev = all(isinstance(a, torch.Tensor) and a.is_cuda for a in arrays)
        if on_dev:
            keep = [a.to(torch.int32).contiguous() for a in arrays]
        else:
            keep = [_host_i32(a) for a in arrays]
        m = int(keep[0].shape[0])
        _check_lengths("Graph", keep, (m, m, n, m))
        h = ctypes.c_void_p()
        st = lib.hm_load_graph(int(n), m, *[_ptr(a) for a in keep], 1 if on_dev else 0,
                               _stream_ptr(stream), ctypes.byref(h))
        check(st, "hm_load_graph")
        self._h = h
        self.n, self.m = int(n), m

    @classmethod
    def with_properties(cls, n: int, src, dst, vprops, eprops, stream=None):
        """A graph whose vertices / arcs carry several int32 properties (arrays [n, nvp], [m, nep])."""
        vp = np.ascontiguousarray(np.asarray(vprops, dtype=np.int32).reshape(n, -1))
        keep = [_host_i32(src), _host_i32(dst)]
        m = int(keep[0].shape[0])
        _check_lengths("Graph.with_properties", keep, (m, m))
        ep = np.ascontiguousarray(np.asarray(eprops, dtype=np.int32).reshape(m, -1))
        h = ctypes.c_void_p()
        check(lib.hm_load_graph_props(int(n), m, _ptr(keep[0]), _ptr(keep[1]), vp.shape[1], _ptr(vp),
                                      ep.shape[1], _ptr(ep), _stream_ptr(stream), ctypes.byref(h)),
              "hm_load_graph_props")
        self = cls.__new__(cls)
        self._h = h
        self.n, self.m = int(n), m
        self.nvp, self.nep = int(vp.shape[1]), int(ep.shape[1])
        return self

    @classmethod
    def from_synth(cls, g, stream=None, device: bool = False):
        if device:
            t = [torch.from_numpy(np.asarray(a)).cuda() for a in (g.src, g.dst, g.vlab, g.elab)]
            return cls(g.n, *t, stream=stream)
        return cls(g.n, g.src, g.dst, g.vlab, g.elab, stream=stream)

    @property
    def handle(self):
        return self._h

    def device_bytes(self) -> int:
        b = ctypes.c_size_t()
        check(lib.hm_graph_info(self._h, None, None, ctypes.byref(b)), "hm_graph_info")
        return int(b.value)

    def export(self) -> dict:
        """Host copies of the built adjacency (offsets int64, lists int32)."""
        n, m = self.n, self.m
        out = {k: np.zeros(n + 1, np.int64) for k in ("out_off", "in_off")}
        out.update({k: np.zeros(max(m, 1), np.int32) for k in ("out_adj", "out_elab", "in_adj", "in_elab")})
        check(lib.hm_graph_export(self._h, *[_ptr(out[k]) for k in
                                             ("out_off", "out_adj", "out_elab", "in_off", "in_adj",
                                              "in_elab")]), "hm_graph_export")
        for k in ("out_adj", "out_elab", "in_adj", "in_elab"):
            out[k] = out[k][:m]
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib.hm_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pattern:
    """A pattern graph after Alg. 1; host-only (needs no GPU)."""

    def __init__(self, k: int, src, dst, vlab, elab, order=None):
        """`order` (optional): the original vertex at each position, replacing Alg. 1's order."""
        keep = [_host_i32(a) for a in (src, dst, vlab, elab)]
        mp = int(keep[0].shape[0])
        _check_lengths("Pattern", keep, (mp, mp, k, mp))
        h = ctypes.c_void_p()
        if order is None:
            st = lib.hm_load_pattern(int(k), int(keep[0].shape[0]), *[_ptr(a) for a in keep],
                                     ctypes.byref(h))
        else:
            o = _host_i32(order)
            if o.shape[0] != int(k):
                raise ValueError("order must list k vertices")
            st = lib.hm_load_pattern_ordered(int(k), int(keep[0].shape[0]), *[_ptr(a) for a in keep],
                                             _ptr(o), ctypes.byref(h))
        check(st, "hm_load_pattern")
        self._h = h
        self.k = int(k)
        self.mp = int(keep[0].shape[0])

    @classmethod
    def from_synth(cls, p, order=None):
        return cls(p.k, p.src, p.dst, p.vlab, p.elab, order=order)

    @classmethod
    def with_properties(cls, g: "Graph", k: int, src, dst, vprops, eprops):
        """A pattern whose vertices / arcs carry g's property tuples ([k, nvp], [mp, nep])."""
        keep = [_host_i32(src), _host_i32(dst)]
        mp = int(keep[0].shape[0])
        _check_lengths("Pattern.with_properties", keep, (mp, mp))
        vp = np.ascontiguousarray(np.asarray(vprops, dtype=np.int32).reshape(k, -1))
        ep = np.ascontiguousarray(np.asarray(eprops, dtype=np.int32).reshape(mp, -1))
        h = ctypes.c_void_p()
        check(lib.hm_load_pattern_props(g.handle, int(k), mp, _ptr(keep[0]), _ptr(keep[1]), _ptr(vp),
                                        _ptr(ep), ctypes.byref(h)), "hm_load_pattern_props")
        self = cls.__new__(cls)
        self._h = h
        self.k, self.mp = int(k), mp
        return self

    @property
    def handle(self):
        return self._h

    @property
    def order(self) -> list[int]:
        out = np.zeros(self.k, np.int32)
        check(lib.hm_pattern_order(self._h, _ptr(out)), "hm_pattern_order")
        return out.tolist()

    def automorphisms(self) -> int:
        """Size of the automorphism group the search uses for symmetry breaking (1: none)."""
        c = ctypes.c_int32()
        check(lib.hm_pattern_automorphisms(self._h, ctypes.byref(c)), "hm_pattern_automorphisms")
        return int(c.value)

    def close(self):
        if getattr(self, "_h", None):
            lib.hm_free_pattern(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def count_matches(g: Graph, p: Pattern, mode: int, stream=None) -> int:
    c = ctypes.c_uint64()
    check(lib.hm_count_matches(g.handle, p.handle, int(mode), ctypes.byref(c), _stream_ptr(stream)),
          "hm_count_matches")
    return int(c.value)


def enumerate_matches(g: Graph, p: Pattern, mode: int, out: torch.Tensor | None = None,
                      capacity: int | None = None, stream=None) -> torch.Tensor:
    """All matches as a CUDA int32 tensor [count, k], rows sorted lexicographically.

    `out` (CUDA int32, >= capacity*k elements) is used if given, and a
    too-small `out` raises HMError(HM_ERR_CAPACITY) carrying the needed count;
    otherwise a buffer of `capacity` rows (default 1<<20) is allocated, and the
    call is repeated with the exact size if it was too small.
    """
    k = p.k
    own = out is None
    if own:
        cap = int(capacity if capacity is not None else 1 << 20)
        if cap < 0:
            raise ValueError("capacity must be >= 0")
        out = torch.empty(max(cap, 1) * k, dtype=torch.int32, device="cuda")
    else:
        cap = _rows_capacity(out, k, capacity)
    c = ctypes.c_uint64()
    st = lib.hm_enumerate_matches(g.handle, p.handle, int(mode), ctypes.c_void_p(out.data_ptr()),
                                  cap, ctypes.byref(c), _stream_ptr(stream))
    if st == binding.HM_ERR_CAPACITY and own:
        need = int(c.value)
        out = torch.empty(max(need, 1) * k, dtype=torch.int32, device="cuda")
        st = lib.hm_enumerate_matches(g.handle, p.handle, int(mode), ctypes.c_void_p(out.data_ptr()),
                                      need, ctypes.byref(c), _stream_ptr(stream))
    check(st, "hm_enumerate_matches", int(c.value))
    return out[: int(c.value) * k].view(int(c.value), k)


def count_matches_part(g: Graph, p: Pattern, mode: int, part: int, nparts: int, stream=None) -> int:
    """Matches seeded by part `part` of `nparts` contiguous ranges of the target's arcs."""
    c = ctypes.c_uint64()
    check(lib.hm_count_matches_part(g.handle, p.handle, int(mode), int(part), int(nparts),
                                    ctypes.byref(c), _stream_ptr(stream)), "hm_count_matches_part")
    return int(c.value)


def enumerate_matches_part(g: Graph, p: Pattern, mode: int, part: int, nparts: int,
                           out: torch.Tensor, stream=None) -> torch.Tensor:
    """Rows of the matches seeded by one arc range, written to `out` (sorted); raises on capacity."""
    k = p.k
    cap = _rows_capacity(out, k, None)
    c = ctypes.c_uint64()
    check(lib.hm_enumerate_matches_part(g.handle, p.handle, int(mode), int(part), int(nparts),
                                        ctypes.c_void_p(out.data_ptr()), cap,
                                        ctypes.byref(c), _stream_ptr(stream)),
          "hm_enumerate_matches_part", int(c.value))
    return out[: int(c.value) * k].view(int(c.value), k)


def _batch_args(patterns, modes):
    n = len(patterns)
    handles = (ctypes.c_void_p * max(n, 1))(*[p.handle.value for p in patterns])
    if isinstance(modes, int):
        modes = [modes] * n
    m = np.ascontiguousarray(np.asarray(modes, dtype=np.int32))
    if m.shape[0] != n:
        raise ValueError("one mode per pattern")
    return n, handles, m


def count_batch(g: Graph, patterns, modes, stream=None) -> list[int]:
    """Counts of many patterns from one edge scan and one persistent extension launch."""
    n, handles, m = _batch_args(patterns, modes)
    out = np.zeros(max(n, 1), np.uint64)
    check(lib.hm_count_batch(g.handle, ctypes.cast(handles, ctypes.c_void_p), _ptr(m), n,
                             ctypes.c_void_p(out.ctypes.data), _stream_ptr(stream)), "hm_count_batch")
    return [int(x) for x in out[:n]]


def enumerate_batch(g: Graph, patterns, modes, counts=None, stream=None) -> list[torch.Tensor]:
    """Sorted rows of many patterns in one pass; sizes the regions with a count pass if needed."""
    n, handles, m = _batch_args(patterns, modes)
    if counts is None:
        counts = count_batch(g, patterns, modes, stream)
    ks = [p.k for p in patterns]
    offs = np.zeros(n + 1, np.uint64)
    for i in range(n):
        offs[i + 1] = offs[i] + np.uint64(counts[i] * ks[i])
    buf = torch.empty(max(int(offs[-1]), 1), dtype=torch.int32, device="cuda")
    got = np.zeros(max(n, 1), np.uint64)
    st = lib.hm_enumerate_batch(g.handle, ctypes.cast(handles, ctypes.c_void_p), _ptr(m), n,
                                ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(offs.ctypes.data),
                                ctypes.c_void_p(got.ctypes.data), _stream_ptr(stream))
    check(st, "hm_enumerate_batch")
    return [buf[int(offs[i]): int(offs[i + 1])].view(int(got[i]), ks[i]) for i in range(n)]


def autotune(g: Graph, patterns, modes, budget_ms: int = 2000, stream=None, cache: str | None = None) -> dict:
    """Tune the launch knobs on the batched count of `patterns` (coordinate descent); install and
    return the best.  With `cache` (a file path), a setting stored for the same graph and pattern
    mix is reused without timing, and a new choice is appended to the file."""
    n, handles, m = _batch_args(patterns, modes)
    t = binding.hm_tuning()
    ms = ctypes.c_float()
    hit = ctypes.c_int32()
    check(lib.hm_autotune_cached(g.handle, ctypes.cast(handles, ctypes.c_void_p), _ptr(m), n, int(budget_ms),
                                 cache.encode() if cache else None, ctypes.byref(t), ctypes.byref(ms),
                                 ctypes.byref(hit), _stream_ptr(stream)), "hm_autotune_cached")
    out = t.as_dict()
    out["ms"] = float(ms.value)
    out["from_cache"] = bool(hit.value)
    return out


class Server:
    """Query server over one resident graph (hm_server_*): submit from any thread, poll for results.

    `slots` dispatcher slots (each a host thread with its own stream) batch the
    waiting queries that the device-memory budget admits; batches of different
    slots overlap on the GPU.
    """

    def __init__(self, g: Graph, slots: int = 4, max_batch: int = 64, mem_budget: int = 0):
        h = ctypes.c_void_p()
        check(lib.hm_server_create(g.handle, int(slots), int(max_batch), int(mem_budget), ctypes.byref(h)),
              "hm_server_create")
        self._h = h
        self._g = g  # the graph must outlive the server
        self._k = {}

    def submit(self, pattern, mode: int, want_rows: bool = True) -> int:
        arrays = [_host_i32(a) for a in (pattern.src, pattern.dst, pattern.vlab, pattern.elab)]
        mp = int(arrays[0].shape[0])
        _check_lengths("Server.submit", arrays, (mp, mp, pattern.k, mp))
        qid = ctypes.c_uint64()
        check(lib.hm_server_submit(self._h, int(pattern.k), int(arrays[0].shape[0]), *[_ptr(a) for a in arrays],
                                   int(mode), 1 if want_rows else 0, ctypes.byref(qid)), "hm_server_submit")
        self._k[int(qid.value)] = int(pattern.k)
        return int(qid.value)

    def result(self, qid: int, wait: bool = True):
        """None while pending; else dict(count, latency_ms, rows_dropped, rows: numpy [n, k] or None).

        A completed query's results are copied out and released on the server.
        """
        done = ctypes.c_int32()
        cnt = ctypes.c_uint64()
        lat = ctypes.c_double()
        dropped = ctypes.c_int32()
        rows = ctypes.POINTER(ctypes.c_int32)()
        nrows = ctypes.c_uint64()
        st = lib.hm_server_poll(self._h, int(qid), 1 if wait else 0, ctypes.byref(done), ctypes.byref(cnt),
                                ctypes.byref(lat), ctypes.byref(dropped), ctypes.byref(rows),
                                ctypes.byref(nrows))
        if not done.value:
            check(st, "hm_server_poll")
            return None
        k = self._k.pop(int(qid))
        out = {"count": int(cnt.value), "latency_ms": float(lat.value), "rows_dropped": bool(dropped.value),
               "rows": None}
        n = int(nrows.value)
        if n:
            out["rows"] = np.ctypeslib.as_array(rows, shape=(n * k,)).copy().reshape(n, k)
        check(lib.hm_server_release(self._h, int(qid)), "hm_server_release")
        check(st, "hm_server_poll")
        return out

    def stats(self) -> dict:
        v = [ctypes.c_uint64() for _ in range(4)]
        check(lib.hm_server_stats(self._h, *[ctypes.byref(x) for x in v]), "hm_server_stats")
        return dict(zip(["batches", "completed", "max_inflight_batches", "rows_dropped"],
                        [int(x.value) for x in v]))

    def close(self):
        if getattr(self, "_h", None):
            lib.hm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def count_matches_rooted(g: Graph, p: Pattern, mode: int, root: int, mask, stream=None) -> int:
    """Count only matches whose image of original pattern vertex `root` is flagged in mask (uint8[n])."""
    if not (isinstance(mask, torch.Tensor) and mask.is_cuda):
        mask = torch.as_tensor(np.asarray(mask, dtype=np.uint8)).cuda()
    mask = mask.to(torch.uint8).contiguous().reshape(-1)
    if int(mask.numel()) != g.n:
        raise ValueError(f"mask has {int(mask.numel())} entries, the graph {g.n} vertices")
    c = ctypes.c_uint64()
    check(lib.hm_count_matches_rooted(g.handle, p.handle, int(mode), int(root),
                                      ctypes.c_void_p(mask.data_ptr()), ctypes.byref(c),
                                      _stream_ptr(stream)), "hm_count_matches_rooted")
    return int(c.value)


def injected_states(g: Graph, p: Pattern, mode: int, stream=None) -> torch.Tensor:
    """The depth-2 states after both validators, as a CUDA int32 tensor [S, 2] (unordered)."""
    cap = max(g.m, 1)
    out = torch.empty(cap * 2, dtype=torch.int32, device="cuda")
    c = ctypes.c_uint64()
    check(lib.hm_injected_states(g.handle, p.handle, int(mode), ctypes.c_void_p(out.data_ptr()), cap,
                                 ctypes.byref(c), _stream_ptr(stream)), "hm_injected_states")
    return out[: int(c.value) * 2].view(int(c.value), 2)


def set_budget(max_ms: int = 0, max_chunks: int = 0):
    check(lib.hm_set_budget(int(max_ms), int(max_chunks)), "hm_set_budget")


def set_timing(enabled: bool):
    check(lib.hm_set_timing(1 if enabled else 0), "hm_set_timing")


def set_counters(enabled: bool):
    """Run instrumented kernels that tally algorithmic bytes (measurement only; slower)."""
    check(lib.hm_set_counters(1 if enabled else 0), "hm_set_counters")


def set_tuning(extend_min_blocks: int = 0, split_min: int = 0, pair_mode: int = 0,
               seeds_per_fetch: int = 0, poll_every: int = 0, leaf_flatten: int = 0,
               arc_filter: int = 0, share_seeds: int = 0, symmetry: int = 0, warps_per_state: int = 0,
               lookahead: int = 0):
    """Set the extension kernel's launch knobs (0 = default; results never change)."""
    t = binding.hm_tuning(int(extend_min_blocks), int(split_min), int(pair_mode),
                          int(seeds_per_fetch), int(poll_every), int(leaf_flatten), int(arc_filter),
                          int(share_seeds), int(symmetry), int(warps_per_state), int(lookahead))
    check(lib.hm_set_tuning(ctypes.byref(t)), "hm_set_tuning")


def get_tuning() -> dict:
    t = binding.hm_tuning()
    check(lib.hm_get_tuning(ctypes.byref(t)), "hm_get_tuning")
    return t.as_dict()


def check_status(g: Graph) -> int:
    """The first out-of-range index the bounds-checked build recorded for g (0 = none),
    cleared by the call; raises HMError(HM_ERR_ARG) in the default build (no checks)."""
    w = ctypes.c_uint64()
    check(lib.hm_check_status(g.handle, ctypes.byref(w)), "hm_check_status")
    return int(w.value)


def last_stats() -> dict:
    s = binding.hm_stats()
    check(lib.hm_last_stats(ctypes.byref(s)), "hm_last_stats")
    return s.as_dict()
