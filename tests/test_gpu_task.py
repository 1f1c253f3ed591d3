"""The task-parallel schedule (k_task: every segment partitioned as soon as its parent is
done, no level barrier) against the CPU oracle, and against the level-by-level schedule
of the same kernels' steps (marked gpu).

The sorted output is unique, so both schedules must give the oracle's bytes for every
key kind, every size class (one tile, a few tiles, a ragged tail, many tiles), long =p
runs (fill items past the inline bound), presorted roots, many root segments, the depth
guard taking segments out of the task kernel, and a withheld tile row that must end in
TSQS_ETIMEOUT through the bounded wait rather than a hang.
"""
import ctypes

import numpy as np
import pytest

from workloads import PATTERNS, int32_pattern, records_u64, rand_u64
from workloads.patterns import batched_segments, batched_keys

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KINDS = {"i32": (1, np.int32), "u32": (2, np.uint32), "f32": (3, np.float32),
         "i64": (4, np.int64), "u64": (5, np.uint64), "f64": (6, np.float64)}


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


def _ctx(T, schedule: int):
    p = T.Plan()
    assert T.lib().tsqs_plan_default(1, 0, ctypes.byref(p)) == 0
    p.schedule = schedule
    return T.Context(p)


def _keys(kind_name: str, n: int, seed: int) -> np.ndarray:
    code, dt = KINDS[kind_name]
    bits = rand_u64(seed, 200 + code, n)
    a = (bits >> np.uint64(32)).astype(np.uint32).view(dt) if np.dtype(dt).itemsize == 4 else bits.view(dt)
    if n > 10:
        a[::5] = a[1]                                   # one long =p run, spread out
    if kind_name in ("f32", "f64") and n > 40:
        sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan], dtype=dt)
        a[7:7 + 6 * (n // 40)] = np.resize(sp, 6 * (n // 40))
    return a


def _dev(a: np.ndarray):
    b = np.ascontiguousarray(a)
    if b.dtype in (np.uint32, np.float32):
        b = b.view(np.int32)
    elif b.dtype in (np.uint64, np.float64):
        b = b.view(np.int64)
    return torch.from_numpy(b.copy()).cuda()


def _oracle(orc, a: np.ndarray, kind: int) -> bytes:
    b = np.ascontiguousarray(a.copy())
    orc.tsqs_sort(b, kind)
    return b.tobytes()


def _sort(T, ctx, a: np.ndarray, kind: int) -> bytes:
    t = _dev(a)
    T.sort_(t, kind=kind, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == T.TSQS_OK
    return t.cpu().numpy().tobytes()


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("kind_name", list(KINDS))
@pytest.mark.parametrize("n", [4097, 5000, 16_385, 65_537, 300_001, 1_000_003])
def test_both_schedules_match_oracle(T, orc, schedule, kind_name, n):
    code = KINDS[kind_name][0]
    a = _keys(kind_name, n, seed=n % 1000 + code)
    ctx = _ctx(T, schedule)
    assert _sort(T, ctx, a, code) == _oracle(orc, a, code)
    ctx.close()


@pytest.mark.parametrize("n", [4097, 70_001, 1_000_003])
def test_records_task_schedule(T, orc, n):
    r = records_u64(n, seed=n)
    ctx = _ctx(T, 2)
    t = torch.from_numpy(r.view(np.int64).copy()).cuda()
    T.sort_(t, records=True, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == T.TSQS_OK
    assert t.cpu().numpy().tobytes() == _oracle(orc, r, 7)
    ctx.close()


@pytest.mark.parametrize("pattern", PATTERNS)
def test_patterns_default_schedule(T, orc, pattern):
    """Seven patterns at 2^22 (the task schedule by default): presorted roots, long =p
    runs (many equals: fill items past the inline bound), organ pipes."""
    n = 1 << 22
    a = int32_pattern(pattern, n, seed=11)
    ctx = T.Context()
    assert _sort(T, ctx, a, 1) == _oracle(orc, a, 1)
    st = ctx.stats()
    assert st["leaf_sorted_keys"] + st["leaf_filled_keys"] + st["presorted_keys"] + st["deep_sorted_keys"] == n
    ctx.close()


def test_few_distinct_values_fill_items(T, orc):
    """Eight distinct values in 3e6 keys: every =p run is far above the inline fill bound,
    so the fills go through the leaf pass as queued items."""
    n = 3_000_000
    a = (rand_u64(5, 9, n) % np.uint64(8)).astype(np.int32)
    ctx = _ctx(T, 2)
    assert _sort(T, ctx, a, 1) == _oracle(orc, a, 1)
    st = ctx.stats()
    assert st["leaf_filled_keys"] >= n - 8 * 4096
    ctx.close()


def test_many_root_segments(T, orc):
    """Root segments of every size class in one call (one warp per root in the task
    init): empty, one element, below and above the on-chip threshold."""
    nseg = 3000
    offs, _, pat = batched_segments(nseg, seed=3, max_log2=16)
    x = batched_keys(offs, pat, seed=3)
    exp = x.copy()
    orc.tsqs_sort_segments(exp, offs, orc.KIND_I32, threads=8)
    ctx = _ctx(T, 2)
    t = torch.from_numpy(x.copy()).cuda()
    d_offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    T.sort_segmented_(t, d_offs, kind=1, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == T.TSQS_OK
    assert t.cpu().numpy().tobytes() == exp.tobytes()
    ctx.close()


def test_task_schedule_at_2e25(T, orc):
    """Schedule 2 past the default bound (2^24): 2^25 keys, a deeper recursion tree."""
    n = 1 << 25
    a = int32_pattern("random", n, seed=4)
    ctx = _ctx(T, 2)
    assert _sort(T, ctx, a, 1) == _oracle(orc, a, 1)
    st = ctx.stats()
    assert st["level_keys"][0] == n and st["levels"] >= 12
    ctx.close()


def test_stats_of_task_schedule(T):
    n = 1 << 22
    a = int32_pattern("random", n, seed=3)
    ctx = T.Context()
    t = torch.from_numpy(a.copy()).cuda()
    T.sort_(t, kind=1, ctx=ctx)
    torch.cuda.synchronize()
    st = ctx.stats()
    assert ctx.status() == 0
    # the root is depth 0; every key is finished by a leaf sort or an =p fill
    assert st["level_keys"][0] == n and st["levels"] >= 9
    assert st["leaf_sorted_keys"] + st["leaf_filled_keys"] == n
    assert st["partition_keys"] == sum(st["level_keys"])
    ctx.close()


@pytest.mark.parametrize("deep", [1, 2, 4])
def test_depth_guard_in_task_schedule(T, orc, deep):
    """Children at depth >= the guard's level leave the task kernel for the bitonic
    sorter (the IF branch the task kernel's last block sets)."""
    n = 1_500_007
    a = int32_pattern("random", n, seed=deep)
    L = T.lib()
    L.tsqs_debug_set_deep_level(deep)
    try:
        ctx = _ctx(T, 2)
        got = _sort(T, ctx, a, 1)
        st = ctx.stats()
        ctx.close()
    finally:
        L.tsqs_debug_set_deep_level(0)
    assert got == _oracle(orc, a, 1)
    assert st["deep_sorted_keys"] > 0
    assert st["leaf_sorted_keys"] + st["leaf_filled_keys"] + st["deep_sorted_keys"] == n


def test_withheld_rows_end_in_timeout(T):
    """The first task segment never publishes its tile rows: every block that claimed
    one of its tiles polls until the spin limit, the sort ends with TSQS_ETIMEOUT, and
    the next sort on the same context is clean."""
    n = 200_003
    a = int32_pattern("random", n, seed=8)
    L = T.lib()
    ctx = _ctx(T, 2)
    L.tsqs_debug_set_spin_limit(2000)
    L.tsqs_debug_withhold_publish(2)
    try:
        t = _dev(a)
        T.sort_(t, kind=1, ctx=ctx)
        torch.cuda.synchronize()
        st = ctx.status()
    finally:
        L.tsqs_debug_withhold_publish(0)
        L.tsqs_debug_set_spin_limit(0)
    assert st == T.TSQS_ETIMEOUT
    t = _dev(a)
    T.sort_(t, kind=1, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert np.array_equal(t.cpu().numpy(), np.sort(a))
    ctx.close()


def test_schedules_agree_on_serving_sizes(T):
    """Request sizes of the serving mix (2^10 .. 2^22) sorted by both schedules on one
    stream, back to back: identical output."""
    rng = np.random.default_rng(1)
    c1, c2 = _ctx(T, 1), _ctx(T, 2)
    for lg in range(10, 23, 2):
        n = int(rng.integers(1 << lg, 2 << lg))
        a = int32_pattern("random", n, seed=lg)
        assert _sort(T, c1, a, 1) == _sort(T, c2, a, 1)
    c1.close()
    c2.close()


@pytest.mark.parametrize("threshold", [512, 1024, 2048])
@pytest.mark.parametrize("kind_name", ["i32", "f64"])
def test_single_tile_segments(T, orc, threshold, kind_name):
    """An on-chip threshold below the task tile: segments that fit in one tile are
    partitioned and finished by one block, with no reservation and no tile count."""
    code = KINDS[kind_name][0]
    n = 400_009
    a = _keys(kind_name, n, seed=threshold + code)
    p = T.Plan()
    assert T.lib().tsqs_plan_default(code, 0, ctypes.byref(p)) == 0
    p.schedule = 2
    p.small_threshold = threshold
    ctx = T.Context(p)
    assert _sort(T, ctx, a, code) == _oracle(orc, a, code)
    st = ctx.stats()
    assert st["leaf_sorted_keys"] + st["leaf_filled_keys"] == n
    ctx.close()


def test_concurrent_task_sorts_on_four_streams(T, orc):
    """Four contexts, four streams, four task-parallel sorts in flight at once (each
    kernel's blocks poll only their own sort's rows): every result equals the oracle's."""
    sizes = [1_000_003, 300_007, 2_000_001, 65_537]
    arrays = [int32_pattern("random", n, seed=40 + i) for i, n in enumerate(sizes)]
    ctxs = [_ctx(T, 2) for _ in sizes]
    streams = [torch.cuda.Stream() for _ in sizes]
    ts = [torch.from_numpy(a.copy()).cuda() for a in arrays]
    torch.cuda.synchronize()
    for rep in range(3):
        for t, a in zip(ts, arrays):
            t.copy_(torch.from_numpy(a))
        torch.cuda.synchronize()
        for t, c, s in zip(ts, ctxs, streams):
            T.sort_(t, kind=1, ctx=c, stream=s)
        torch.cuda.synchronize()
        for t, a, c in zip(ts, arrays, ctxs):
            assert c.status() == T.TSQS_OK
            assert t.cpu().numpy().tobytes() == _oracle(orc, a, 1)
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("kind_name", ["i32", "u32", "f32"])
def test_small_input_leaf_every_item_size(T, orc, kind_name):
    """Below 2^20 keys the task graph's leaf pass takes the small-input leaf kernel (256
    threads x 16 keys per item): root segments of 1 .. 4096 keys in one call are all leaf
    items of that kernel, each compared with the oracle."""
    code, dt = KINDS[kind_name]
    sizes = list(range(1, 4097, 9)) + [4095, 4096]
    offs = np.zeros(len(sizes) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(sizes)
    n = int(offs[-1])
    assert n <= 1 << 20
    a = _keys(kind_name, n, seed=77 + code)
    exp = np.ascontiguousarray(a.copy())
    orc.tsqs_sort_segments(exp, offs, code, threads=8)
    ctx = T.Context()
    t = _dev(a)
    d_offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    T.sort_segmented_(t, d_offs, kind=code, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == T.TSQS_OK
    got = t.cpu().numpy().view(dt)
    if got.tobytes() != exp.tobytes():
        bad = [k for k in range(len(sizes))
               if got[offs[k]:offs[k + 1]].tobytes() != exp[offs[k]:offs[k + 1]].tobytes()]
        raise AssertionError(f"{len(bad)} items differ, sizes {[sizes[k] for k in bad[:5]]}")
    ctx.close()


@pytest.mark.parametrize("kind_name", list(KINDS))
@pytest.mark.parametrize("n", [5000, 300_001])
def test_task_schedule_unaligned_bases(T, orc, kind_name, n):
    """Arrays whose base is aligned to the element but not to 16 bytes: the task kernel's
    tiles start below the segment, the buffer's ends take scalar loads, and the =p fills
    write a scalar head and tail around their 16-byte body."""
    code, dt = KINDS[kind_name]
    es = np.dtype(dt).itemsize
    a = _keys(kind_name, n, seed=n % 97 + code)
    a[::3] = a[2]                                   # long =p runs for the fills
    exp = _oracle(orc, a, code)
    ctx = _ctx(T, 2)
    for off in range(1, 16 // es):
        big = _dev(np.concatenate([a[:off], a, a[:4]]))   # room before and after
        view = big[off:off + n]
        assert view.data_ptr() % 16 != 0
        T.sort_(view, kind=code, ctx=ctx)
        torch.cuda.synchronize()
        assert ctx.status() == T.TSQS_OK
        assert view.cpu().numpy().tobytes() == exp
        # the elements around the view are untouched
        around = big.cpu().numpy()
        assert around[:off].tobytes() == np.ascontiguousarray(a[:off]).view(around.dtype).tobytes()
        assert around[off + n:].tobytes() == np.ascontiguousarray(a[:4]).view(around.dtype).tobytes()
    ctx.close()


@pytest.mark.parametrize("kind_name", ["i32", "f64"])
def test_task_schedule_host_array(T, orc, kind_name):
    """A pinned host array sorted through tsqs_sort_host: below the size bound the task
    schedule writes its =p fills and leaf sorts straight into the mapped host array."""
    code, dt = KINDS[kind_name]
    n = 700_001
    a = _keys(kind_name, n, seed=31 + code)
    exp = _oracle(orc, a, code)
    h = torch.from_numpy(np.ascontiguousarray(a).view(np.int32 if np.dtype(dt).itemsize == 4 else np.int64).copy()).pin_memory()
    assert T.lib().tsqs_sort_host(ctypes.c_void_p(h.data_ptr()), n, np.dtype(dt).itemsize, code, None) == 0
    assert h.numpy().tobytes() == exp


@pytest.mark.parametrize("kind_name", ["i64", "f64", "rec"])
def test_depth_guard_in_task_schedule_wide_keys(T, orc, kind_name):
    """The cooperative depth guard for 8-byte keys and records (the largest tile buffer):
    with the guard at depth 2, most keys reach it, and the output equals the oracle's."""
    n = 600_007
    if kind_name == "rec":
        a = records_u64(n, seed=17)
        code = 7
        t = torch.from_numpy(a.view(np.int64).copy()).cuda()
    else:
        code = KINDS[kind_name][0]
        a = _keys(kind_name, n, seed=19 + code)
        t = _dev(a)
    exp = _oracle(orc, a, code)
    L = T.lib()
    L.tsqs_debug_set_deep_level(2)
    try:
        ctx = _ctx(T, 2)
        T.sort_(t, kind=code, ctx=ctx)
        torch.cuda.synchronize()
        assert ctx.status() == T.TSQS_OK
        st = ctx.stats()
        ctx.close()
    finally:
        L.tsqs_debug_set_deep_level(0)
    assert t.cpu().numpy().tobytes() == exp
    assert st["deep_sorted_keys"] > n // 2
