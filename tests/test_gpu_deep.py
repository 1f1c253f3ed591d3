"""Depth guard on the GPU: with the guard's level forced low, segments that would
recurse deeper are sorted by the bitonic fallback; every result must still equal the
oracle's, and the statistics must show the fallback ran."""
import ctypes

import numpy as np
import pytest

from workloads import PATTERNS, int32_pattern, records_u64, floats_normal_specials

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


@pytest.fixture
def deep(T):
    def set_level(level):
        T.lib().tsqs_debug_set_deep_level(level)
    yield set_level
    T.lib().tsqs_debug_set_deep_level(0)


def _dev(a):
    b = np.ascontiguousarray(a)
    if b.dtype == np.uint64:
        b = b.view(np.int64)
    return torch.from_numpy(b.copy()).cuda()


def _oracle(orc, a, kind):
    b = np.ascontiguousarray(a.copy())
    orc.tsqs_sort(b, kind)
    return b


@pytest.mark.parametrize("level", [1, 2, 5])
@pytest.mark.parametrize("n", [5000, 70_001, 2_000_003])
def test_deep_fallback_random_int32(T, orc, deep, level, n):
    deep(level)
    a = int32_pattern("random", n, seed=level + n)
    ctx = T.Context()
    t = _dev(a)
    T.sort_(t, kind=1, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert t.cpu().numpy().tobytes() == _oracle(orc, a, 1).tobytes()
    st = ctx.stats()
    if (n >> level) > 3 * 4096:          # segments at the guard's depth still above 4096
        assert st["deep_sorted_keys"] > 0
    assert st["leaf_sorted_keys"] + st["leaf_filled_keys"] + st["presorted_keys"] + st["deep_sorted_keys"] == n
    ctx.close()


@pytest.mark.parametrize("pattern", [p for p in PATTERNS if p not in ("sorted", "stair_steps")])
def test_deep_fallback_patterns(T, orc, deep, pattern):
    deep(2)
    n = 300_007
    a = int32_pattern(pattern, n, seed=9)
    t = _dev(a)
    T.sort_(t, kind=1)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    assert t.cpu().numpy().tobytes() == _oracle(orc, a, 1).tobytes()


def test_deep_fallback_records_floats_i64(T, orc, deep):
    deep(1)
    r = records_u64(150_001, seed=4)
    t = torch.from_numpy(r.view(np.int64).copy()).cuda()
    T.sort_(t, records=True)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    assert t.cpu().numpy().view(np.uint64).reshape(-1, 2).tobytes() == _oracle(orc, r, 7).tobytes()
    f = floats_normal_specials(200_003, seed=5)
    t = _dev(f)
    T.sort_(t, kind=3)
    torch.cuda.synchronize()
    assert t.cpu().numpy().view(np.float32).tobytes() == _oracle(orc, f, 3).tobytes()
    x = (np.arange(100_000, dtype=np.int64) * 7919) % 100_003 - 50_000
    t = _dev(x)
    T.sort_(t, kind=4)
    torch.cuda.synchronize()
    assert t.cpu().numpy().tobytes() == _oracle(orc, x, 4).tobytes()


def test_deep_fallback_segmented_and_host(T, orc, deep):
    deep(1)
    rng = np.random.default_rng(12)
    sizes = rng.integers(1, 40_000, 60)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    a = rng.integers(-2**31, 2**31 - 1, int(offs[-1])).astype(np.int32)
    t = _dev(a)
    T.sort_segmented_(t, torch.from_numpy(offs).cuda(), kind=1)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    exp = a.copy()
    orc.tsqs_sort_segments(exp, offs.astype(np.uint64), 1, threads=4)
    assert t.cpu().numpy().tobytes() == exp.tobytes()
    # host array: the fallback's result reaches the mapped output
    h = torch.from_numpy(a.copy()).pin_memory()
    assert T.lib().tsqs_sort_host(ctypes.c_void_p(h.data_ptr()), len(a), 4, 1, None) == 0
    assert h.numpy().tobytes() == _oracle(orc, a, 1).tobytes()
