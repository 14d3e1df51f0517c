"""CPU oracle for labelled directed subgraph matching -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never imports,
links or calls anything here, and this package imports nothing from the
product package: the two share no code.  The only module both sides use is
``synth`` (seeded input arrays, no matching arithmetic).

Contents
  * ``oracle.c`` -- plain backtracking matcher from the empty mapping, in C
    with POSIX threads (Sec. II-A, Eqs. 1-3).  Built with gcc into
    ``oracle/_build/liboracle.so`` by :func:`build`.
  * :mod:`oracle.bruteforce` -- every injective map on tiny inputs (pure Python).
  * :mod:`oracle.steps` -- the method's own host steps written out plainly from
    the paper: Alg. 1 (structural reordering), Alg. 2 (vertex validator) and
    Alg. 3 with the edge loop of the HiPerMotif algorithm (edge validator and
    state injection), used to check the CUDA path's intermediate results.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MONO, INDUCED = 0, 1


def build(src: str | None = None, out: str | None = None, extra_flags=()) -> str:
    """Compile the C oracle with gcc (-O2, pthreads) and return the .so path."""
    src = src or os.path.join(_HERE, "oracle.c")
    out = out or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = f"{out}.tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
           *extra_flags, src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.og_graph_new.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i32p,
                                 ctypes.POINTER(ctypes.c_void_p)]
    lib.og_graph_new.restype = ctypes.c_int
    lib.og_graph_free.argtypes = [ctypes.c_void_p]
    lib.og_graph_free.restype = None
    lib.og_match.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p,
                             i32p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(i32p)]
    lib.og_match.restype = ctypes.c_int
    lib.og_rows_free.argtypes = [ctypes.c_void_p]
    lib.og_rows_free.restype = None
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library; `path` selects another build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            src = os.path.join(_HERE, "oracle.c")
            if (not os.path.exists(_LIB_PATH)
                    or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src)):
                build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
        return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _c32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


class OracleGraph:
    """The oracle's own copy of a target graph (sorted out/in lists with labels)."""

    def __init__(self, n, src, dst, vlab, elab, lib=None):
        self._lib = lib or load()
        self.n = int(n)
        self._keep = [_c32(src), _c32(dst), _c32(vlab), _c32(elab)]
        h = ctypes.c_void_p()
        rc = self._lib.og_graph_new(self.n, len(self._keep[0]), *[_p32(a) for a in self._keep],
                                    ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"oracle rejected the graph (code {rc})")
        self._h = h
        self._keep = None

    @classmethod
    def from_synth(cls, g, lib=None):
        return cls(g.n, g.src, g.dst, g.vlab, g.elab, lib=lib)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.og_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def match(self, pattern, mode: int, *, rows: bool = True, threads: int | None = None,
              root_mask: np.ndarray | None = None):
        """Return (count, rows) for `pattern` (a synth.Pattern or any object with k/src/dst/vlab/elab).

        rows is an int64-free int32 array [count, k] sorted lexicographically, or None.
        root_mask (uint8[n]) keeps only maps whose image of original vertex 0 is flagged.
        """
        k = int(pattern.k)
        ps, pd, pv, pe = (_c32(pattern.src), _c32(pattern.dst), _c32(pattern.vlab),
                          _c32(pattern.elab))
        if threads is None:
            threads = os.cpu_count() or 1
        mask_ptr = None
        if root_mask is not None:
            rm = np.ascontiguousarray(root_mask, dtype=np.uint8)
            assert rm.shape[0] == self.n
            mask_ptr = rm.ctypes.data_as(ctypes.c_void_p)
        cnt = ctypes.c_uint64(0)
        out = ctypes.POINTER(ctypes.c_int32)()
        rc = self._lib.og_match(self._h, k, len(ps), _p32(ps), _p32(pd), _p32(pv), _p32(pe),
                                int(mode), int(threads), mask_ptr, 1 if rows else 0,
                                ctypes.byref(cnt), ctypes.byref(out))
        if rc != 0:
            raise ValueError(f"oracle rejected the pattern (code {rc})")
        count = int(cnt.value)
        if not rows:
            return count, None
        arr = np.ctypeslib.as_array(out, shape=(max(count, 1) * k,))[: count * k].copy()
        self._lib.og_rows_free(ctypes.cast(out, ctypes.c_void_p))
        return count, arr.reshape(count, k)


def match(graph, pattern, mode: int, **kw):
    """One-shot convenience: build the oracle graph, match, free."""
    og = OracleGraph.from_synth(graph)
    try:
        return og.match(pattern, mode, **kw)
    finally:
        og.close()
