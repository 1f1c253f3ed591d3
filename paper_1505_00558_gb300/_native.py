"""ctypes binding of libtsqs.so: the C-ABI entry points under the same names.

Argument marshalling only.  Every step of the sort runs in the library's CUDA
kernels; there is no Python or CPU fallback.  If the library is missing this module
raises at load time.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtsqs.so")

TSQS_I32, TSQS_U32, TSQS_F32, TSQS_I64, TSQS_U64, TSQS_F64, TSQS_U64_U64_REC = 1, 2, 3, 4, 5, 6, 7
TSQS_OK, TSQS_EINVAL, TSQS_ENOMEM, TSQS_ECUDA, TSQS_ETIMEOUT, TSQS_EINTERNAL = 0, 1, 2, 3, 4, 5
STATUS_NAMES = {0: "TSQS_OK", 1: "TSQS_EINVAL", 2: "TSQS_ENOMEM", 3: "TSQS_ECUDA",
                4: "TSQS_ETIMEOUT", 5: "TSQS_EINTERNAL"}
ELEM_SIZE = {1: 4, 2: 4, 3: 4, 4: 8, 5: 8, 6: 8, 7: 16}


class Plan(ctypes.Structure):
    _fields_ = [("tile_items", ctypes.c_int32), ("small_threshold", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("sample_count", ctypes.c_int32),
                ("offset_mode", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_uint32), ("max_frontier", ctypes.c_uint32),
                ("partition_keys", ctypes.c_uint64), ("leaf_sorted_keys", ctypes.c_uint64),
                ("leaf_filled_keys", ctypes.c_uint64), ("leaf_items", ctypes.c_uint64),
                ("presorted_keys", ctypes.c_uint64), ("deep_sorted_keys", ctypes.c_uint64),
                ("level_keys_count", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("level_keys", ctypes.c_uint64 * 64)]

    def as_dict(self):
        d = {k: int(getattr(self, k)) for k, _ in self._fields_ if k not in ("level_keys", "pad")}
        d["level_keys"] = [int(self.level_keys[i]) for i in range(self.level_keys_count)]
        return d


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("done", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("batch_id", ctypes.c_uint32),
                ("batch_size", ctypes.c_uint32)]


# name -> (restype, argtypes); every function the header declares
_vp, _sz, _i, _u32, _u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
_pu64 = ctypes.POINTER(ctypes.c_uint64)
SIGNATURES = {
    "tsqs_sort": (_i, [_vp, _sz, _sz, _i, _vp]),
    "tsqs_sort_segmented": (_i, [_vp, _sz, _vp, _sz, _sz, _i, _vp]),
    "tsqs_sort_host": (_i, [_vp, _sz, _sz, _i, _vp]),
    "tsqs_sort_noalloc": (_i, [_vp, _sz, _sz, _i, _vp]),
    "tsqs_sort_wide": (_i, [_vp, _sz, _sz, _sz, _i, _vp]),
    "tsqs_free_storage": (None, []),
    "tsqs_last_device_status": (_i, [_vp]),
    "tsqs_ctx_create": (_vp, [ctypes.POINTER(Plan)]),
    "tsqs_ctx_destroy": (None, [_vp]),
    "tsqs_ctx_sort": (_i, [_vp, _vp, _sz, _sz, _i, _vp]),
    "tsqs_ctx_sort_segmented": (_i, [_vp, _vp, _sz, _vp, _sz, _sz, _i, _vp]),
    "tsqs_graph_sort_segmented": (_i, [_vp, _vp, _sz, _vp, _sz, _sz, _i, _vp,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "tsqs_graph_exec_destroy": (None, [_vp, _vp]),
    "tsqs_ctx_reserve": (_i, [_vp, _sz, _sz, _sz]),
    "tsqs_ctx_scratch_bytes": (_sz, [_vp]),
    "tsqs_ctx_device_status": (_i, [_vp, _vp]),
    "tsqs_ctx_stats": (_i, [_vp, _vp, ctypes.POINTER(Stats)]),
    "tsqs_ctx_set_plan": (_i, [_vp, ctypes.POINTER(Plan)]),
    "tsqs_ctx_get_plan": (_i, [_vp, ctypes.POINTER(Plan)]),
    "tsqs_ctx_sort_host_stream": (_i, [_vp, _vp, _vp, _vp, _sz, _sz, _i, _vp, _vp]),
    "tsqs_scratch_bytes_for": (_sz, [_sz, _sz, _sz, ctypes.POINTER(Plan)]),
    "tsqs_plan_default": (_i, [_i, _sz, ctypes.POINTER(Plan)]),
    "tsqs_ctx_sort_timed": (_i, [_vp, _vp, _sz, _sz, _i, _vp, ctypes.POINTER(ctypes.c_float),
                                 _pu64, _i, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_float)]),
    "tsqs_debug_pivot": (_i, [_vp, _sz, _sz, _i, _u64, _u64, _i, _u64, _pu64, _vp, _vp]),
    "tsqs_debug_partition": (_i, [_vp, _vp, _sz, _sz, _i, _vp, _sz, _vp, _vp, _vp]),
    "tsqs_debug_small_sort": (_i, [_vp, _sz, _sz, _i, _vp, _sz, _vp]),
    "tsqs_debug_set_spin_limit": (None, [_u32]),
    "tsqs_debug_set_deep_level": (None, [_u32]),
    "tsqs_debug_set_leaf_defer": (None, [_u32]),
    "tsqs_debug_withhold_publish": (None, [_i]),
    "tsqs_plan_autotune": (_i, [_i, _sz, _sz, _vp, ctypes.POINTER(Plan)]),
    "tsqs_plan_cache_save": (_i, [ctypes.c_char_p]),
    "tsqs_plan_cache_load": (_i, [ctypes.c_char_p]),
    "tsqs_server_create": (_vp, [_sz, _i, _i]),
    "tsqs_server_submit": (_i, [_vp, _vp, _sz, _sz, _i, _pu64]),
    "tsqs_server_progress": (_i, [_vp]),
    "tsqs_server_poll": (_i, [_vp, _u64, ctypes.POINTER(Result)]),
    "tsqs_server_drain": (_i, [_vp]),
    "tsqs_server_destroy": (None, [_vp]),
}

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Loads libtsqs.so (built by __graft_entry__.build() or build.py).  Raises if the
    library or any declared entry point is missing: there is no fallback."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libtsqs.so not built ({LIB_PATH}); run "
                                   "python -c 'import __graft_entry__ as g; g.build()'")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)
