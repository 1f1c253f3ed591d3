"""Argument checking at the C-ABI boundary (host logic only: every call here is
rejected, or is a no-op, before any device call, so it runs without a GPU).  The
boundary's contract: a kind/size mismatch, a NULL array for a non-empty sort, a base
not aligned to its element, or a size over a limit returns TSQS_EINVAL and queues
nothing; 0 or 1 element returns TSQS_OK."""
import ctypes
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def T():
    if shutil.which("nvcc") is None and not os.path.exists(
            os.path.join(ROOT, "paper_1505_00558_gb300", "libtsqs.so")):
        pytest.skip("nvcc not available to build libtsqs.so")
    from paper_1505_00558_gb300 import build
    build.build()
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


@pytest.fixture(scope="module")
def host_buf():
    # a 16-byte-aligned host address; the calls below never dereference it
    raw = ctypes.create_string_buffer(4096)
    base = (ctypes.addressof(raw) + 15) & ~15
    return raw, base


def test_core_sort_arguments(T, host_buf):
    L = T.lib()
    _, p = host_buf
    vp = ctypes.c_void_p
    assert L.tsqs_sort(vp(p), 100, 8, T.TSQS_I32, None) == T.TSQS_EINVAL       # size != kind
    assert L.tsqs_sort(vp(p), 100, 4, 99, None) == T.TSQS_EINVAL               # no such kind
    assert L.tsqs_sort(None, 100, 4, T.TSQS_I32, None) == T.TSQS_EINVAL        # NULL, n > 1
    assert L.tsqs_sort(vp(p + 4), 100, 8, T.TSQS_I64, None) == T.TSQS_EINVAL   # misaligned
    assert L.tsqs_sort(vp(p + 8), 100, 16, T.TSQS_U64_U64_REC, None) == T.TSQS_EINVAL
    assert L.tsqs_sort(vp(p + 2), 100, 4, T.TSQS_F32, None) == T.TSQS_EINVAL
    assert L.tsqs_sort(None, 1, 4, T.TSQS_I32, None) == T.TSQS_OK              # nothing to do
    assert L.tsqs_sort(vp(p), 0, 8, T.TSQS_F64, None) == T.TSQS_OK
    assert L.tsqs_sort_segmented(vp(p), 10, None, 3, 4, T.TSQS_I32, None) == T.TSQS_EINVAL


def test_context_and_noalloc_arguments(T, host_buf):
    L = T.lib()
    _, p = host_buf
    vp = ctypes.c_void_p
    assert L.tsqs_ctx_sort(None, vp(p), 10, 4, T.TSQS_I32, None) == T.TSQS_EINVAL
    ctx = vp(L.tsqs_ctx_create(None))
    assert ctx.value
    assert L.tsqs_ctx_sort(ctx, vp(p), 10, 4, T.TSQS_I64, None) == T.TSQS_EINVAL
    assert L.tsqs_ctx_sort(ctx, vp(p), 1, 4, T.TSQS_I32, None) == T.TSQS_OK
    g = ctypes.c_void_p(None)
    f = L.tsqs_graph_sort_segmented
    assert f(ctx, vp(p), 10, None, 0, 4, T.TSQS_I32, None, None) == T.TSQS_EINVAL          # no handle
    assert f(ctx, vp(p), 10, None, 0, 8, T.TSQS_I32, None, ctypes.byref(g)) == T.TSQS_EINVAL
    assert f(ctx, vp(p), 10, None, 3, 4, T.TSQS_I32, None, ctypes.byref(g)) == T.TSQS_EINVAL  # nseg, no offsets
    assert f(None, vp(p), 10, None, 0, 4, T.TSQS_I32, None, ctypes.byref(g)) == T.TSQS_EINVAL
    assert f(ctx, vp(p), 1, None, 0, 4, T.TSQS_I32, None, ctypes.byref(g)) == T.TSQS_OK     # nothing to do
    assert g.value is None
    bogus = ctypes.c_void_p(p)                  # not a graph of this context
    assert f(ctx, vp(p), 10, None, 0, 4, T.TSQS_I32, None, ctypes.byref(bogus)) == T.TSQS_EINVAL
    L.tsqs_graph_exec_destroy(ctx, bogus)       # ignored
    L.tsqs_ctx_destroy(ctx)
    over = (16 << 20) // 4 + 1                     # TSQS_NOALLOC_MAX_BYTES is 16 MiB
    assert L.tsqs_sort_noalloc(vp(p), over, 4, T.TSQS_I32, None) == T.TSQS_EINVAL
    assert L.tsqs_sort_noalloc(vp(p), 100, 8, T.TSQS_I32, None) == T.TSQS_EINVAL
    assert L.tsqs_sort_noalloc(vp(p), 1, 4, T.TSQS_I32, None) == T.TSQS_OK
    # sizes whose byte count wraps around 2^64 are over the limit too
    huge = (1 << 64) // 4 + 1
    assert L.tsqs_sort_noalloc(vp(p), huge, 4, T.TSQS_I32, None) == T.TSQS_EINVAL
    assert L.tsqs_sort_noalloc(vp(p), (1 << 64) // 16 + 3, 16, T.TSQS_U64_U64_REC, None) == T.TSQS_EINVAL


def test_wide_and_host_stream_arguments(T, host_buf):
    L = T.lib()
    _, p = host_buf
    vp = ctypes.c_void_p
    assert L.tsqs_sort_wide(vp(p), 100, 10, 0, T.TSQS_I32, None) == T.TSQS_EINVAL   # not x4
    assert L.tsqs_sort_wide(vp(p), 100, 12, 4, T.TSQS_I64, None) == T.TSQS_EINVAL   # key past end
    assert L.tsqs_sort_wide(vp(p), 100, 16, 0, T.TSQS_U64_U64_REC, None) == T.TSQS_EINVAL
    assert L.tsqs_sort_wide(vp(p), 1 << 31, 16, 0, T.TSQS_I32, None) == T.TSQS_EINVAL
    assert L.tsqs_sort_wide(vp(p), 1, 16, 0, T.TSQS_I32, None) == T.TSQS_OK
    ctx = vp(L.tsqs_ctx_create(None))
    ins = (ctypes.c_void_p * 2)(p, p)
    sizes = (ctypes.c_size_t * 2)(64, 64)
    f = L.tsqs_ctx_sort_host_stream
    assert f(ctx, ins, None, sizes, 2, 8, T.TSQS_I32, None, None) == T.TSQS_EINVAL
    assert f(ctx, ins, None, (ctypes.c_size_t * 2)(64, 1 << 31), 2, 4, T.TSQS_I32, None, None) == T.TSQS_EINVAL
    assert f(ctx, (ctypes.c_void_p * 2)(p, None), None, sizes, 2, 4, T.TSQS_I32, None, None) == T.TSQS_EINVAL
    assert f(ctx, None, None, None, 2, 4, T.TSQS_I32, None, None) == T.TSQS_EINVAL
    assert f(None, ins, None, sizes, 2, 4, T.TSQS_I32, None, None) == T.TSQS_EINVAL
    assert f(ctx, None, None, None, 0, 4, T.TSQS_I32, None, None) == T.TSQS_OK
    L.tsqs_ctx_destroy(ctx)


def test_plan_defaults_and_scratch_bounds(T):
    L = T.lib()
    for kind in (T.TSQS_I32, T.TSQS_F64, T.TSQS_U64_U64_REC):
        plan = T.Plan()
        assert L.tsqs_plan_default(kind, 1 << 20, ctypes.byref(plan)) == T.TSQS_OK
        assert plan.sample_count % 2 == 1 and 1 <= plan.sample_count <= 63
        assert 512 <= plan.small_threshold <= 4096
        es = {T.TSQS_I32: 4, T.TSQS_F64: 8, T.TSQS_U64_U64_REC: 16}[kind]
        a = L.tsqs_scratch_bytes_for(1 << 20, 1, es, ctypes.byref(plan))
        b = L.tsqs_scratch_bytes_for(1 << 22, 1, es, ctypes.byref(plan))
        c = L.tsqs_scratch_bytes_for(1 << 22, 5000, es, ctypes.byref(plan))
        assert (1 << 20) * es < a < b <= c        # at least the second buffer, growing with n and nseg


def test_schedule_decides_the_task_tables(T):
    """The task-parallel schedule's tables are part of the scratch exactly when a sort of
    that size takes it: below the 2^24 bound by default (schedule 0), at any size with
    schedule 2, never with schedule 1 or look-back offsets (no GPU needed)."""
    L = T.lib()

    def need(n, schedule, offset_mode=0):
        p = T.Plan()
        assert L.tsqs_plan_default(T.TSQS_I32, 0, ctypes.byref(p)) == T.TSQS_OK
        p.schedule = schedule
        p.offset_mode = offset_mode
        return L.tsqs_scratch_bytes_for(n, 1, 4, ctypes.byref(p))

    for n in (1 << 16, 1_000_000, 1 << 24):
        assert need(n, 0) > need(n, 1)            # task tables below the bound
        assert need(n, 0) == need(n, 2)
        assert need(n, 0, offset_mode=1) == need(n, 1)
    for n in ((1 << 24) + 1, 1 << 26):
        assert need(n, 0) == need(n, 1)           # level by level above it
        assert need(n, 2) > need(n, 1)
    # the tables stay a small fraction of the second buffer
    assert need(1 << 24, 0) - need(1 << 24, 1) < (1 << 24) * 4
