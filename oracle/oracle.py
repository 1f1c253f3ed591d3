"""ctypes binding of the C oracle (test infrastructure; see the package docstring).

Arrays are numpy arrays: 4-byte kinds as int32/uint32/float32, 8-byte kinds as
int64/uint64/float64, records as a (n, 2) uint64 array (key, payload) or any
C-contiguous buffer of n * 16 bytes.  Every call works in place on a copy the
caller owns; nothing here touches a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsqs_oracle.c")
_LIB = os.path.join(_HERE, "libtsqs_oracle.so")
_STD_SRC = os.path.join(_HERE, "std_sort_ref.cpp")
_STD_LIB = os.path.join(_HERE, "libstd_sort_ref.so")

KIND_I32, KIND_U32, KIND_F32, KIND_I64, KIND_U64, KIND_F64, KIND_REC = 1, 2, 3, 4, 5, 6, 7
PIVOT_TIERED, PIVOT_RANDOM = 0, 1
STATE_NAMES = ("state1", "2L", "2R", "3L", "3R", "init_special", "exit_state1")

_ELEM = {KIND_I32: 4, KIND_U32: 4, KIND_F32: 4, KIND_I64: 8, KIND_U64: 8, KIND_F64: 8,
         KIND_REC: 16}


class _Cfg(ctypes.Structure):
    _fields_ = [("ins_threshold", ctypes.c_int), ("pivot_policy", ctypes.c_int),
                ("random_samples", ctypes.c_int), ("med3_below", ctypes.c_int),
                ("med5_below", ctypes.c_int), ("ninther_below", ctypes.c_int),
                ("seed", ctypes.c_uint64)]


class _Stats(ctypes.Structure):
    _fields_ = [("cmps", ctypes.c_uint64), ("moves", ctypes.c_uint64),
                ("swaps", ctypes.c_uint64), ("stages", ctypes.c_uint64),
                ("ins_parts", ctypes.c_uint64), ("max_depth", ctypes.c_uint64),
                ("tar_peak", ctypes.c_uint64), ("state_entries", ctypes.c_uint64 * 7)]

    def as_dict(self) -> dict:
        d = {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "state_entries"}
        d["states"] = {STATE_NAMES[i]: int(self.state_entries[i]) for i in range(7)}
        return d


@dataclass
class OracleCfg:
    """Oracle configuration; defaults are the readings listed in the C header."""
    ins_threshold: int = 16
    pivot_policy: int = PIVOT_TIERED
    random_samples: int = 1
    med3_below: int = 70
    med5_below: int = 800
    ninther_below: int = 40000
    seed: int = 1

    def _c(self) -> _Cfg:
        return _Cfg(self.ins_threshold, self.pivot_policy, self.random_samples,
                    self.med3_below, self.med5_below, self.ninther_below, self.seed)


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc -O2 (portable C11, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _LIB)
    if force or not os.path.exists(_STD_LIB) or os.path.getmtime(_STD_LIB) < os.path.getmtime(_STD_SRC):
        tmp = _STD_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _STD_SRC])
        os.replace(tmp, _STD_LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            vp, sz, i, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64
            ps, pc = ctypes.POINTER(_Stats), ctypes.POINTER(_Cfg)
            L.orc_tsqs_sort.argtypes = [vp, sz, i, pc, ps]
            L.orc_tsqs_sort_rows.argtypes = [vp, sz, sz, i, pc, ps]
            L.orc_tsqs_sort_segments.argtypes = [vp, vp, sz, i, i]
            L.orc_classical_sort.argtypes = [vp, sz, i, u64, ps]
            L.orc_juggle_sort.argtypes = [vp, sz, i, u64, ps]
            L.orc_median3.argtypes = [vp, sz, sz, sz, i, ps]
            L.orc_choose_pivot.argtypes = [vp, sz, i, pc, ps]
            L.orc_choose_pivot.restype = ctypes.c_longlong
            L.orc_lower_median.argtypes = [vp, sz, i, vp]
            L.orc_three_way_split.argtypes = [vp, vp, sz, i, vp, ctypes.POINTER(sz),
                                              ctypes.POINTER(sz), ctypes.POINTER(sz)]
            L.orc_compare.argtypes = [vp, vp, i]
            L.orc_wide_sort.argtypes = [vp, sz, sz, sz, i, ctypes.POINTER(u64), ctypes.POINTER(u64)]
            L.orc_elem_size.argtypes = [i]
            L.orc_elem_size.restype = sz
            _lib = L
    return _lib


def _check(a: np.ndarray, kind: int) -> int:
    if not a.flags.c_contiguous:
        raise ValueError("oracle arrays must be C-contiguous")
    es = _ELEM[kind]
    if a.nbytes % es:
        raise ValueError("buffer size is not a multiple of the element size")
    return a.nbytes // es


def tsqs_sort(a: np.ndarray, kind: int, cfg: OracleCfg | None = None) -> dict:
    """Triple State QuickSort of ``a`` in place; returns the counters."""
    n = _check(a, kind)
    st = _Stats()
    c = (cfg or OracleCfg())._c()
    if lib().orc_tsqs_sort(a.ctypes.data, n, kind, ctypes.byref(c), ctypes.byref(st)):
        raise RuntimeError("oracle sort failed")
    return st.as_dict()


def tsqs_sort_rows(a: np.ndarray, kind: int, cfg: OracleCfg | None = None) -> dict:
    """Sorts every row of a 2-D array (or (rows, n, 2) record array) independently."""
    rows = a.shape[0]
    total = _check(a, kind)
    n = total // rows if rows else 0
    st = _Stats()
    c = (cfg or OracleCfg())._c()
    if lib().orc_tsqs_sort_rows(a.ctypes.data, rows, n, kind, ctypes.byref(c), ctypes.byref(st)):
        raise RuntimeError("oracle sort failed")
    return st.as_dict()


def wide_sort(a: np.ndarray, elem_size: int, key_offset: int, kind: int) -> dict:
    """Late-swap sort (Section VIII.H) of the raw bytes of ``a``, viewed as elements of
    elem_size bytes with a key of ``kind`` at key_offset; returns the move and cycle
    counts."""
    if not a.flags.c_contiguous or a.nbytes % elem_size:
        raise ValueError("wide arrays must be C-contiguous whole elements")
    mv, cy = ctypes.c_uint64(), ctypes.c_uint64()
    if lib().orc_wide_sort(a.ctypes.data, a.nbytes // elem_size, elem_size, key_offset, kind,
                           ctypes.byref(mv), ctypes.byref(cy)):
        raise RuntimeError("oracle wide sort failed")
    return {"moves": mv.value, "cycles": cy.value}


def tsqs_sort_segments(a: np.ndarray, offsets: np.ndarray, kind: int, threads: int = 1) -> None:
    _check(a, kind)
    offs = np.ascontiguousarray(offsets, dtype=np.uint64)
    if lib().orc_tsqs_sort_segments(a.ctypes.data, offs.ctypes.data, len(offs) - 1, kind, threads):
        raise RuntimeError("oracle segmented sort failed")


def classical_sort(a: np.ndarray, kind: int, seed: int = 1) -> dict:
    n = _check(a, kind)
    st = _Stats()
    lib().orc_classical_sort(a.ctypes.data, n, kind, seed, ctypes.byref(st))
    return st.as_dict()


def juggle_sort(a: np.ndarray, kind: int, seed: int = 1) -> dict:
    n = _check(a, kind)
    st = _Stats()
    lib().orc_juggle_sort(a.ctypes.data, n, kind, seed, ctypes.byref(st))
    return st.as_dict()


def median3(a: np.ndarray, kind: int, i0: int = 0, i1: int = 1, i2: int = 2) -> tuple[int, dict]:
    _check(a, kind)
    st = _Stats()
    o = lib().orc_median3(a.ctypes.data, i0, i1, i2, kind, ctypes.byref(st))
    return o, st.as_dict()


def choose_pivot(a: np.ndarray, kind: int, cfg: OracleCfg | None = None) -> tuple[int, dict]:
    """Pivot selection of Section III.H alone on the part ``a`` (in place: the tier's
    samples end sorted); returns the pivot index and the counters."""
    n = _check(a, kind)
    st = _Stats()
    c = (cfg or OracleCfg())._c()
    pi = lib().orc_choose_pivot(a.ctypes.data, n, kind, ctypes.byref(c), ctypes.byref(st))
    if pi < 0:
        raise ValueError("choose_pivot needs n >= 3 and a known key kind")
    return int(pi), st.as_dict()


def lower_median(keys: np.ndarray, kind: int) -> np.ndarray:
    s = _check(keys, kind)
    out = np.zeros(_ELEM[kind], dtype=np.uint8)
    if lib().orc_lower_median(keys.ctypes.data, s, kind, out.ctypes.data):
        raise RuntimeError("lower_median failed")
    return out.view(keys.dtype)


def three_way_split(a: np.ndarray, kind: int, pivot) -> tuple[np.ndarray, int, int, int]:
    n = _check(a, kind)
    out = np.empty_like(a)
    pv = np.ascontiguousarray(np.asarray(pivot, dtype=a.dtype).reshape(-1)[: (2 if kind == KIND_REC else 1)])
    nlt, neq, ngt = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    lib().orc_three_way_split(a.ctypes.data, out.ctypes.data, n, kind, pv.ctypes.data,
                              ctypes.byref(nlt), ctypes.byref(neq), ctypes.byref(ngt))
    return out, nlt.value, neq.value, ngt.value


_std_lib = None


def std_sort_i32(a: np.ndarray) -> None:
    """std::sort of an int32 array in place (the library reference timed beside the
    oracle; single-threaded on the calling thread)."""
    global _std_lib
    if a.dtype != np.int32 or not a.flags.c_contiguous:
        raise ValueError("std_sort_i32 takes a C-contiguous int32 array")
    with _lock:
        if _std_lib is None:
            build()
            _std_lib = ctypes.CDLL(_STD_LIB)
            _std_lib.orc_std_sort_i32.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    _std_lib.orc_std_sort_i32(a.ctypes.data, len(a))


def compare(x, y, kind: int) -> int:
    xa = np.ascontiguousarray(x)
    ya = np.ascontiguousarray(y)
    return lib().orc_compare(xa.ctypes.data, ya.ctypes.data, kind)
