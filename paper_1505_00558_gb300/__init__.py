"""GB300-native three-way partition sort (Triple State QuickSort, arXiv 1505.00558).

The compute path is libtsqs.so (hand-written CUDA for sm_103a behind a C-ABI, see
include/tsqs.h).  This package is the thin Python side: the C entry points under the
same names (``paper_1505_00558_gb300.tsqs_sort`` etc.) plus tensor helpers that only
marshal ``data_ptr()``, sizes and the current CUDA stream.  PyTorch provides device
memory and streams; it computes nothing here.
"""
from __future__ import annotations

import ctypes

from . import _native
from ._native import (  # noqa: F401
    TSQS_I32, TSQS_U32, TSQS_F32, TSQS_I64, TSQS_U64, TSQS_F64, TSQS_U64_U64_REC,
    TSQS_OK, TSQS_EINVAL, TSQS_ENOMEM, TSQS_ECUDA, TSQS_ETIMEOUT, TSQS_EINTERNAL,
    STATUS_NAMES, ELEM_SIZE, Plan, Stats, Result, SIGNATURES, lib,
)


class TsqsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)}")
        self.code = code


def __getattr__(name):
    # tsqs_* entry points resolve to the C functions themselves
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)


def _check(rc: int, what: str) -> None:
    if rc != TSQS_OK:
        raise TsqsError(rc, what)


# ------------------------------------------------------------------------------
# tensor helpers (marshalling only)
# ------------------------------------------------------------------------------

def key_kind_of(t, records: bool = False) -> int:
    """Key kind of a tensor: int32/uint32/float32/int64/uint64/float64, or records
    when ``records`` is set (a C-contiguous (n, 2) 64-bit tensor: key, payload)."""
    import torch
    if records:
        if t.dim() != 2 or t.shape[1] != 2 or t.element_size() != 8:
            raise ValueError("records must be an (n, 2) tensor of 64-bit elements")
        return TSQS_U64_U64_REC
    m = {torch.int32: TSQS_I32, torch.float32: TSQS_F32, torch.int64: TSQS_I64,
         torch.float64: TSQS_F64}
    if hasattr(torch, "uint32"):
        m[torch.uint32] = TSQS_U32
    if hasattr(torch, "uint64"):
        m[torch.uint64] = TSQS_U64
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def _stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _geom(t, kind: int):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    es = ELEM_SIZE[kind]
    n = t.numel() * t.element_size() // es
    return ctypes.c_void_p(t.data_ptr()), n, es


def sort_(t, *, kind: int | None = None, records: bool = False, stream=None, ctx=None):
    """Sorts tensor ``t`` in place on its device (asynchronous on ``stream``)."""
    kind = kind or key_kind_of(t, records)
    p, n, es = _geom(t, kind)
    s = ctypes.c_void_p(_stream_handle(stream))
    if ctx is None:
        _check(lib().tsqs_sort(p, n, es, kind, s), "tsqs_sort")
    else:
        _check(lib().tsqs_ctx_sort(ctx.handle, p, n, es, kind, s), "tsqs_ctx_sort")
    return t


def sort_wide_(t, elem_size: int, key_offset: int, key_kind: int, *, stream=None):
    """Sorts the wide elements held in tensor ``t`` (any dtype; ``t.numel() *
    t.element_size()`` bytes = nmemb * elem_size) by the key of ``key_kind`` at
    ``key_offset`` bytes inside each element, stably, in place on its device."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("sort_wide_ needs a contiguous CUDA tensor")
    nbytes = t.numel() * t.element_size()
    if elem_size <= 0 or nbytes % elem_size:
        raise ValueError("tensor size is not a whole number of elements")
    s = ctypes.c_void_p(_stream_handle(stream))
    _check(lib().tsqs_sort_wide(ctypes.c_void_p(t.data_ptr()), nbytes // elem_size, elem_size,
                                key_offset, key_kind, s), "tsqs_sort_wide")
    return t


def sort_segmented_(t, offsets, *, kind: int | None = None, records: bool = False,
                    stream=None, ctx=None):
    """Sorts every segment [offsets[s], offsets[s+1]) of ``t`` in place.  ``offsets`` is
    a CUDA int64 tensor of nseg + 1 non-decreasing offsets."""
    kind = kind or key_kind_of(t, records)
    p, n, es = _geom(t, kind)
    if not offsets.is_cuda or offsets.element_size() != 8 or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous CUDA int64 tensor")
    nseg = offsets.numel() - 1
    total = n
    s = ctypes.c_void_p(_stream_handle(stream))
    po = ctypes.c_void_p(offsets.data_ptr())
    if ctx is None:
        rc = lib().tsqs_sort_segmented(p, total, po, nseg, es, kind, s)
    else:
        rc = lib().tsqs_ctx_sort_segmented(ctx.handle, p, total, po, nseg, es, kind, s)
    _check(rc, "tsqs_sort_segmented")
    return t


def last_device_status(stream=None) -> int:
    return lib().tsqs_last_device_status(ctypes.c_void_p(_stream_handle(stream)))


def free_storage() -> None:
    lib().tsqs_free_storage()


class Context:
    """An independent sorter (own scratch and graphs)."""

    def __init__(self, plan: Plan | None = None):
        self.handle = ctypes.c_void_p(lib().tsqs_ctx_create(ctypes.byref(plan) if plan else None))
        if not self.handle.value:
            raise TsqsError(TSQS_ENOMEM, "tsqs_ctx_create")

    def close(self):
        if self.handle and self.handle.value:
            lib().tsqs_ctx_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, n: int, nseg: int, elem_size: int):
        _check(lib().tsqs_ctx_reserve(self.handle, n, nseg, elem_size), "tsqs_ctx_reserve")

    def scratch_bytes(self) -> int:
        return lib().tsqs_ctx_scratch_bytes(self.handle)

    def status(self, stream=None) -> int:
        return lib().tsqs_ctx_device_status(self.handle, ctypes.c_void_p(_stream_handle(stream)))

    def stats(self, stream=None) -> dict:
        st = Stats()
        _check(lib().tsqs_ctx_stats(self.handle, ctypes.c_void_p(_stream_handle(stream)),
                                    ctypes.byref(st)), "tsqs_ctx_stats")
        return st.as_dict()

    def plan(self) -> Plan:
        p = Plan()
        _check(lib().tsqs_ctx_get_plan(self.handle, ctypes.byref(p)), "tsqs_ctx_get_plan")
        return p

    def set_plan(self, plan: Plan):
        _check(lib().tsqs_ctx_set_plan(self.handle, ctypes.byref(plan)), "tsqs_ctx_set_plan")

    def sort_host_stream(self, ins, outs=None, *, kind: int | None = None, records: bool = False,
                         stream=None) -> list:
        """Sorts a sequence of contiguous CPU tensors through the GPU with uploads and
        downloads overlapping the sorts (tsqs_ctx_sort_host_stream).  ``outs`` None sorts
        in place; otherwise outs[i] (same size as ins[i]) receives ins[i] sorted.
        Returns each item's device status; raises on a nonzero return."""
        ins = list(ins)
        outs = ins if outs is None else list(outs)
        if len(outs) != len(ins):
            raise ValueError("ins and outs differ in length")
        kind = kind or (key_kind_of(ins[0], records) if ins else TSQS_I32)
        es = ELEM_SIZE[kind]
        cnt = len(ins)
        p_in = (ctypes.c_void_p * max(1, cnt))()
        p_out = (ctypes.c_void_p * max(1, cnt))()
        sizes = (ctypes.c_size_t * max(1, cnt))()
        for i, (a, b) in enumerate(zip(ins, outs)):
            if a.is_cuda or b.is_cuda or not a.is_contiguous() or not b.is_contiguous():
                raise ValueError("expected contiguous CPU tensors")
            nb = a.numel() * a.element_size()
            if b.numel() * b.element_size() != nb:
                raise ValueError("input and output sizes differ")
            p_in[i], p_out[i], sizes[i] = a.data_ptr(), b.data_ptr(), nb // es
        st = (ctypes.c_int * max(1, cnt))()
        rc = lib().tsqs_ctx_sort_host_stream(self.handle, p_in, p_out, sizes, cnt, es, kind,
                                             ctypes.c_void_p(_stream_handle(stream)), st)
        _check(rc, "tsqs_ctx_sort_host_stream")
        return [st[i] for i in range(cnt)]

    def graph_sort_segmented(self, t, offsets, graph_exec=None, *, kind: int | None = None,
                             records: bool = False, stream=None):
        """tsqs_graph_sort_segmented: sorts the segments of ``t`` (``offsets`` a CUDA int64
        tensor of nseg + 1 offsets, or None for one segment) through a caller-held graph.
        Pass the handle returned by an earlier call to update and relaunch that graph;
        returns the handle (a cudaGraphExec_t as int, None if nothing was sorted)."""
        kind = kind or key_kind_of(t, records)
        p, n, es = _geom(t, kind)
        if offsets is not None:
            if not offsets.is_cuda or offsets.element_size() != 8 or not offsets.is_contiguous():
                raise ValueError("offsets must be a contiguous CUDA int64 tensor")
            po, nseg = ctypes.c_void_p(offsets.data_ptr()), offsets.numel() - 1
        else:
            po, nseg = None, 0
        h = ctypes.c_void_p(graph_exec)
        _check(lib().tsqs_graph_sort_segmented(self.handle, p, n, po, nseg, es, kind,
                                               ctypes.c_void_p(_stream_handle(stream)),
                                               ctypes.byref(h)), "tsqs_graph_sort_segmented")
        return h.value

    def graph_destroy(self, graph_exec) -> None:
        lib().tsqs_graph_exec_destroy(self.handle, ctypes.c_void_p(graph_exec))

    def sort_timed(self, t, *, kind: int | None = None, records: bool = False, stream=None,
                   max_levels: int = 256):
        """Level-by-level run of the same kernels with CUDA events around each
        partition launch; returns (partition ms per level, keys per level, leaf ms)."""
        kind = kind or key_kind_of(t, records)
        p, n, es = _geom(t, kind)
        ms = (ctypes.c_float * max_levels)()
        lms = (ctypes.c_float * max_levels)()
        keys = (ctypes.c_uint64 * max_levels)()
        lv = ctypes.c_int(0)
        _check(lib().tsqs_ctx_sort_timed(self.handle, p, n, es, kind,
                                         ctypes.c_void_p(_stream_handle(stream)), ms, keys,
                                         max_levels, ctypes.byref(lv), lms), "tsqs_ctx_sort_timed")
        L = min(lv.value, max_levels)
        return [ms[i] for i in range(L)], [int(keys[i]) for i in range(L)], [lms[i] for i in range(L)]
