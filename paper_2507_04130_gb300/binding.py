"""ctypes binding of libhipermotif.so: the C ABI of include/hipermotif.h, same names.

Argument marshalling only -- every step of the matching path runs in the CUDA
library.  Importing this module loads the library and raises ImportError if
it has not been built (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

from . import _build

HM_OK, HM_ERR_ARG, HM_ERR_SELF_LOOP, HM_ERR_DUP_EDGE, HM_ERR_PATTERN = 0, 1, 2, 3, 4
HM_ERR_OOM, HM_ERR_CAPACITY, HM_ERR_BUDGET, HM_ERR_CUDA, HM_ERR_NO_DEVICE = 5, 6, 7, 8, 9
HM_MONO, HM_INDUCED = 0, 1
HM_MAX_K = 20
HM_STATIC_MAX_ARCS = 3702528

#: every function include/hipermotif.h declares
EXPORTED = [
    "hm_status_str", "hm_load_graph", "hm_free_graph", "hm_graph_info", "hm_check_status", "hm_graph_export",
    "hm_graph_export_groups",
    "hm_load_pattern", "hm_free_pattern", "hm_pattern_order", "hm_count_matches",
    "hm_enumerate_matches", "hm_count_matches_rooted", "hm_count_matches_part",
    "hm_enumerate_matches_part", "hm_injected_states", "hm_set_budget",
    "hm_last_stats", "hm_set_timing", "hm_set_counters", "hm_count_matches_static",
    "hm_set_tuning", "hm_get_tuning", "hm_count_batch", "hm_enumerate_batch", "hm_autotune",
    "hm_server_create", "hm_server_submit", "hm_server_poll", "hm_server_release",
    "hm_server_stats", "hm_server_destroy", "hm_load_graph_props", "hm_load_pattern_props",
    "hm_load_pattern_ordered", "hm_pattern_automorphisms", "hm_autotune_cached",
]


class hm_stats(ctypes.Structure):
    _fields_ = [
        ("seeds_scanned", ctypes.c_uint64),
        ("states_injected", ctypes.c_uint64),
        ("tasks_donated", ctypes.c_uint64),
        ("chunks", ctypes.c_uint64),
        ("matches", ctypes.c_uint64),
        ("ms_edge_scan", ctypes.c_float),
        ("ms_overlap", ctypes.c_float),
        ("ms_extend", ctypes.c_float),
        ("ms_sort", ctypes.c_float),
        ("extend_grid", ctypes.c_int32),
        ("extend_block", ctypes.c_int32),
        ("kernel_launches", ctypes.c_uint32),
        ("pad", ctypes.c_uint32),
        ("bytes_edge_scan", ctypes.c_uint64),
        ("bytes_overlap", ctypes.c_uint64),
        ("bytes_extend", ctypes.c_uint64),
        ("candidates", ctypes.c_uint64),
        ("level_chunks", ctypes.c_uint64 * HM_MAX_K),
        ("level_candidates", ctypes.c_uint64 * HM_MAX_K),
        ("model_bytes_edge_scan", ctypes.c_uint64),
        ("model_bytes_overlap", ctypes.c_uint64),
        ("model_bytes_extend", ctypes.c_uint64),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name.startswith("level_") else v
        return out



class hm_tuning(ctypes.Structure):
    _fields_ = [
        ("extend_min_blocks", ctypes.c_int32),
        ("split_min", ctypes.c_int32),
        ("pair_mode", ctypes.c_int32),
        ("seeds_per_fetch", ctypes.c_int32),
        ("poll_every", ctypes.c_int32),
        ("leaf_flatten", ctypes.c_int32),
        ("arc_filter", ctypes.c_int32),
        ("share_seeds", ctypes.c_int32),
        ("symmetry", ctypes.c_int32),
        ("warps_per_state", ctypes.c_int32),
        ("lookahead", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_st = ctypes.c_int
_pvp = ctypes.POINTER(ctypes.c_void_p)
_pu64 = ctypes.POINTER(ctypes.c_uint64)

_SIGS = {
    "hm_status_str": (ctypes.c_char_p, [_st]),
    "hm_load_graph": (_st, [_i32, _i64, _vp, _vp, _vp, _vp, ctypes.c_int, _vp, _pvp]),
    "hm_free_graph": (None, [_vp]),
    "hm_check_status": (_st, [_vp, ctypes.POINTER(ctypes.c_uint64)]),
    "hm_graph_info": (_st, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64),
                            ctypes.POINTER(ctypes.c_size_t)]),
    "hm_graph_export": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hm_graph_export_groups": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hm_load_pattern": (_st, [_i32, _i32, _vp, _vp, _vp, _vp, _pvp]),
    "hm_load_pattern_ordered": (_st, [_i32, _i32, _vp, _vp, _vp, _vp, _vp, _pvp]),
    "hm_load_graph_props": (_st, [_i32, _i64, _vp, _vp, _i32, _vp, _i32, _vp, _vp, _pvp]),
    "hm_load_pattern_props": (_st, [_vp, _i32, _i32, _vp, _vp, _vp, _vp, _pvp]),
    "hm_free_pattern": (None, [_vp]),
    "hm_pattern_order": (_st, [_vp, _vp]),
    "hm_count_matches": (_st, [_vp, _vp, ctypes.c_int, _pu64, _vp]),
    "hm_enumerate_matches": (_st, [_vp, _vp, ctypes.c_int, _vp, _u64, _pu64, _vp]),
    "hm_count_matches_rooted": (_st, [_vp, _vp, ctypes.c_int, _i32, _vp, _pu64, _vp]),
    "hm_injected_states": (_st, [_vp, _vp, ctypes.c_int, _vp, _u64, _pu64, _vp]),
    "hm_count_matches_part": (_st, [_vp, _vp, ctypes.c_int, _i32, _i32, _pu64, _vp]),
    "hm_enumerate_matches_part": (_st, [_vp, _vp, ctypes.c_int, _i32, _i32, _vp, _u64, _pu64, _vp]),
    "hm_set_budget": (_st, [_u64, _u64]),
    "hm_last_stats": (_st, [ctypes.POINTER(hm_stats)]),
    "hm_set_timing": (_st, [ctypes.c_int]),
    "hm_set_counters": (_st, [ctypes.c_int]),
    "hm_count_matches_static": (_st, [_vp, _vp, ctypes.c_int, _pu64, _vp]),
    "hm_set_tuning": (_st, [ctypes.POINTER(hm_tuning)]),
    "hm_count_batch": (_st, [_vp, _vp, _vp, _i32, _vp, _vp]),
    "hm_server_create": (_st, [_vp, _i32, _i32, _u64, _pvp]),
    "hm_server_submit": (_st, [_vp, _i32, _i32, _vp, _vp, _vp, _vp, _i32, _i32, _pu64]),
    "hm_server_poll": (_st, [_vp, _u64, _i32, ctypes.POINTER(_i32), _pu64, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(_i32), ctypes.POINTER(ctypes.POINTER(_i32)), _pu64]),
    "hm_server_release": (_st, [_vp, _u64]),
    "hm_server_stats": (_st, [_vp, _pu64, _pu64, _pu64, _pu64]),
    "hm_server_destroy": (None, [_vp]),
    "hm_autotune": (_st, [_vp, _vp, _vp, _i32, ctypes.c_uint32, ctypes.POINTER(hm_tuning),
                          ctypes.POINTER(ctypes.c_float), _vp]),
    "hm_enumerate_batch": (_st, [_vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp]),
    "hm_get_tuning": (_st, [ctypes.POINTER(hm_tuning)]),
    "hm_pattern_automorphisms": (_st, [_vp, ctypes.POINTER(_i32)]),
    "hm_autotune_cached": (_st, [_vp, _vp, _vp, _i32, ctypes.c_uint32, ctypes.c_char_p,
                                 ctypes.POINTER(hm_tuning), ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(_i32), _vp]),
}


def _load():
    # HM_CHECK=1 in the environment loads the bounds-checked build instead
    # (paper_2507_04130_gb300._build.build(check=True) makes it)
    checked = os.environ.get("HM_CHECK", "0") == "1"
    path = _build.LIB_CHECK if checked else _build.LIB
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            + ("(python -c 'from paper_2507_04130_gb300 import _build; _build.build(check=True)')" if checked
               else "(python -c 'import __graft_entry__ as g; g.build()')"))
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class HMError(RuntimeError):
    def __init__(self, status: int, where: str, count: int | None = None):
        self.status = int(status)
        self.count = count
        msg = lib.hm_status_str(self.status).decode()
        super().__init__(f"{where}: {msg} (status {self.status})")


def check(status: int, where: str, count: int | None = None):
    if status != HM_OK:
        raise HMError(status, where, count)
