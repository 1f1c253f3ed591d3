"""The level loop's pause for a leaf pass: with the leaf queue's pause threshold forced
down, the graph leaves its level loop whenever too many leaf items wait, sorts them,
and resumes the levels.  Every result must still equal the oracle's (Section III's
recursion on the two outer parts, in any order).  The sorts run on contexts whose plan
asks for the level-by-level schedule (the task-parallel one has no level loop)."""
import ctypes

import numpy as np
import pytest

from workloads import int32_pattern, records_u64, floats_normal_specials

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


def level_ctx(T):
    p = T.Plan()
    assert T.lib().tsqs_plan_default(1, 0, ctypes.byref(p)) == 0
    p.schedule = 1
    return T.Context(p)


@pytest.fixture
def defer(T):
    def set_defer(items):
        T.lib().tsqs_debug_set_leaf_defer(items)
    yield set_defer
    T.lib().tsqs_debug_set_leaf_defer(0)


def _oracle(orc, a, kind):
    b = np.ascontiguousarray(a.copy())
    orc.tsqs_sort(b, kind)
    return b


@pytest.mark.parametrize("items", [1, 3, 40])
@pytest.mark.parametrize("n", [9_000, 300_001, 3_000_017])
def test_pause_random_int32(T, orc, defer, items, n):
    defer(items)
    a = int32_pattern("random", n, seed=items + n)
    ctx = level_ctx(T)
    t = torch.from_numpy(a.copy()).cuda()
    T.sort_(t, kind=1, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert t.cpu().numpy().tobytes() == _oracle(orc, a, 1).tobytes()
    st = ctx.stats()
    assert st["leaf_sorted_keys"] + st["leaf_filled_keys"] + st["presorted_keys"] + st["deep_sorted_keys"] == n
    ctx.close()


@pytest.mark.parametrize("pattern", ["many_equals", "organ_pipe", "nearly_sorted", "reversed"])
def test_pause_patterns(T, orc, defer, pattern):
    defer(2)
    a = int32_pattern(pattern, 500_009, seed=5)
    ctx = level_ctx(T)
    t = torch.from_numpy(a.copy()).cuda()
    T.sort_(t, kind=1, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert t.cpu().numpy().tobytes() == _oracle(orc, a, 1).tobytes()
    ctx.close()


def test_pause_records_floats(T, orc, defer):
    defer(1)
    ctx = level_ctx(T)
    r = records_u64(200_003, seed=8)
    t = torch.from_numpy(r.view(np.int64).copy()).cuda()
    T.sort_(t, records=True, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert t.cpu().numpy().view(np.uint64).reshape(-1, 2).tobytes() == _oracle(orc, r, 7).tobytes()
    f = floats_normal_specials(400_001, seed=9)
    t = torch.from_numpy(f.copy()).cuda()
    T.sort_(t, kind=3, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert t.cpu().numpy().view(np.float32).tobytes() == _oracle(orc, f, 3).tobytes()
    ctx.close()


def test_pause_segmented_host_and_timed(T, orc, defer):
    defer(2)
    rng = np.random.default_rng(21)
    sizes = rng.integers(0, 60_000, 80)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    a = rng.integers(-2**31, 2**31 - 1, int(offs[-1])).astype(np.int32)
    ctx = level_ctx(T)
    t = torch.from_numpy(a.copy()).cuda()
    T.sort_segmented_(t, torch.from_numpy(offs).cuda(), kind=1, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ctx.close()
    exp = a.copy()
    orc.tsqs_sort_segments(exp, offs.astype(np.uint64), 1, threads=4)
    assert t.cpu().numpy().tobytes() == exp.tobytes()
    # host array, written through the mapped output (default context: at this size the
    # task-parallel schedule)
    b = int32_pattern("random", 1_000_003, seed=22)
    h = torch.from_numpy(b.copy()).pin_memory()
    assert T.lib().tsqs_sort_host(ctypes.c_void_p(h.data_ptr()), len(b), 4, 1, None) == 0
    assert h.numpy().tobytes() == _oracle(orc, b, 1).tobytes()
    # host-driven run of the same kernels: its per-level leaf launch takes the pause
    ctx = level_ctx(T)
    c = torch.from_numpy(b.copy()).cuda()
    ms, keys, lms = ctx.sort_timed(c, kind=1)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert c.cpu().numpy().tobytes() == _oracle(orc, b, 1).tobytes()
    ctx.close()
