"""CUDA path vs the CPU oracle (marked gpu).

The sorted output under a total order is unique, so every comparison with the oracle
is bit-exact.  Step-level tests check each kernel alone: the pivot kernel against the
lower median of the sample it reports, one partition level against the plain
three-way split, the leaf sorter at every size up to the on-chip threshold.
Full-size workloads are checked against the plain definition (a library sort) and
by properties that hold at any size.
"""
import ctypes

import numpy as np
import pytest

from workloads import (PATTERNS, int32_pattern, records_u64, floats_normal_specials,
                       rand_u64, total_order_key_f32)
from workloads.patterns import batched_segments, batched_keys

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KINDS = {  # name: (kind code, numpy dtype, torch dtype)
    "i32": (1, np.int32, torch.int32), "u32": (2, np.uint32, None), "f32": (3, np.float32, torch.float32),
    "i64": (4, np.int64, torch.int64), "u64": (5, np.uint64, None), "f64": (6, np.float64, torch.float64),
}


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


def to_dev(a: np.ndarray):
    """numpy -> CUDA tensor holding the same bytes (uint kinds travel as signed)."""
    b = np.ascontiguousarray(a)
    if b.dtype == np.uint32:
        b = b.view(np.int32)
    elif b.dtype == np.uint64:
        b = b.view(np.int64)
    return torch.from_numpy(b.copy()).cuda()


def from_dev(t, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def gpu_sort(T, a: np.ndarray, kind: int) -> np.ndarray:
    t = to_dev(a)
    T.sort_(t, kind=kind)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    return from_dev(t, a.dtype).reshape(a.shape)


def oracle_sort(orc, a: np.ndarray, kind: int) -> np.ndarray:
    b = np.ascontiguousarray(a.copy())
    orc.tsqs_sort(b, kind)
    return b


def random_keys(kind_name: str, n: int, seed: int) -> np.ndarray:
    code, dt, _ = KINDS[kind_name]
    bits = rand_u64(seed, 100 + code, n)
    if np.dtype(dt).itemsize == 4:
        a = (bits >> np.uint64(32)).astype(np.uint32).view(dt)
    else:
        a = bits.view(dt)
    if n > 10:                                        # duplicates and equal runs
        a[::7] = a[3]
    if kind_name in ("f32", "f64") and n > 20:        # specials, NaNs of both signs
        sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan], dtype=dt)
        k = min(6 * (n // 40), n - 5)
        a[5:5 + k] = np.resize(sp, k)
    return a


SIZES = [0, 1, 2, 3, 5, 31, 64, 100, 1000, 4095, 4096, 4097, 8191, 8192, 8193, 65537, 100_003]


@pytest.mark.parametrize("kind_name", list(KINDS))
@pytest.mark.parametrize("n", SIZES)
def test_sort_matches_oracle_all_kinds(T, orc, kind_name, n):
    code = KINDS[kind_name][0]
    a = random_keys(kind_name, n, seed=n + 1)
    got = gpu_sort(T, a, code)
    exp = oracle_sort(orc, a, code)
    assert got.tobytes() == exp.tobytes()


@pytest.mark.parametrize("n", [1, 2, 4095, 4096, 4097, 50_001, 300_007])
def test_records_match_oracle(T, orc, n):
    r = records_u64(n, seed=n)
    t = torch.from_numpy(r.view(np.int64).copy()).cuda()
    T.sort_(t, records=True)
    torch.cuda.synchronize()
    got = t.cpu().numpy().view(np.uint64)
    exp = oracle_sort(orc, r, 7)
    assert got.tobytes() == exp.tobytes()


@pytest.mark.parametrize("pattern", PATTERNS)
def test_patterns_match_oracle(T, orc, pattern):
    n = (1 << 20) + 123
    a = int32_pattern(pattern, n, seed=5)
    assert gpu_sort(T, a, 1).tobytes() == oracle_sort(orc, a, 1).tobytes()


def test_c1_one_million_uniform_matches_oracle(T, orc):
    a = int32_pattern("random", 1_000_000, seed=1)
    assert gpu_sort(T, a, 1).tobytes() == oracle_sort(orc, a, 1).tobytes()


def test_floats_specials_match_oracle(T, orc):
    x = floats_normal_specials(400_000, seed=3, special_frac=0.01)
    assert gpu_sort(T, x, 3).tobytes() == oracle_sort(orc, x, 3).tobytes()


def test_degenerate_inputs(T, orc):
    for a in (np.zeros(70_000, np.int32),
              np.full(70_000, -5, np.int32),
              np.tile(np.array([2 ** 31 - 1, -2 ** 31], np.int32), 40_000),
              np.repeat(np.arange(3, dtype=np.int32), 30_001)[::-1].copy()):
        assert gpu_sort(T, a, 1).tobytes() == oracle_sort(orc, a, 1).tobytes()


def test_unaligned_base(T, orc):
    """base aligned to the element but not to 16 bytes: the head and tail of every
    segment take the scalar path."""
    n = 200_001
    a = int32_pattern("random", n + 3, seed=9)
    for off in (1, 2, 3):
        t = to_dev(a)
        view = t[off:off + n]
        T.sort_(view, kind=1)
        torch.cuda.synchronize()
        got = from_dev(t, np.int32)
        exp = a.copy()
        exp[off:off + n] = oracle_sort(orc, a[off:off + n], 1)
        assert got.tobytes() == exp.tobytes()


def test_deterministic_and_stream(T):
    a = int32_pattern("random", 3_000_000, seed=4)
    s = torch.cuda.Stream()
    outs = []
    for _ in range(2):
        t = to_dev(a)
        with torch.cuda.stream(s):
            T.sort_(t, kind=1, stream=s)
        s.synchronize()
        outs.append(t.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], np.sort(a))


# ------------------------------------------------------------------------------
# step-level tests
# ------------------------------------------------------------------------------

def test_pivot_kernel_is_lower_median_of_its_sample(T, orc):
    n = 1_000_003
    a = int32_pattern("random", n, seed=6)
    t = to_dev(a)
    for (b, e, S) in [(0, n, 31), (17, 100_017, 63), (5000, 9100, 15), (123, 4220, 31),
                      (40, 140, 63), (7, 38, 63), (3, 4, 31)]:
        pos = (ctypes.c_uint64 * S)()
        S = min(S, e - b) - (1 - min(S, e - b) % 2)
        piv = np.zeros(1, np.int32)
        rc = T.lib().tsqs_debug_pivot(ctypes.c_void_p(t.data_ptr()), n, 4, 1, b, e, S, 77, pos,
                                      ctypes.c_void_p(piv.ctypes.data), None)
        assert rc == 0
        p = np.array([pos[i] for i in range(S)], dtype=np.int64)
        m = e - b
        k = np.arange(S)
        lo = b + (m * k) // S
        hi = b + (m * (k + 1)) // S
        assert ((p >= lo) & (p < hi)).all(), "sample outside its stratum"
        assert orc.lower_median(a[p].copy(), 1)[0] == piv[0]


@pytest.mark.parametrize("kind_name", ["i32", "f64"])
def test_partition_level_matches_three_way_split(T, orc, kind_name):
    code, dt, _ = KINDS[kind_name]
    n = 400_000
    a = random_keys(kind_name, n, seed=12)
    a[::3] = a[10]
    cuts = np.unique(np.concatenate([[0, n], (rand_u64(3, 3, 40) % np.uint64(n)).astype(np.int64)]))
    offs = cuts.astype(np.int64)
    nseg = len(offs) - 1
    piv = np.array([a[offs[s] + (offs[s + 1] - offs[s]) // 3] for s in range(nseg)], dtype=dt)
    src = to_dev(a)
    dst = to_dev(np.zeros_like(a))
    d_offs = torch.from_numpy(offs).cuda()
    d_piv = to_dev(piv)
    d_cnt = torch.zeros(2 * nseg, dtype=torch.int64, device="cuda")
    rc = T.lib().tsqs_debug_partition(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                      n, a.itemsize, code, ctypes.c_void_p(d_offs.data_ptr()), nseg,
                                      ctypes.c_void_p(d_piv.data_ptr()), ctypes.c_void_p(d_cnt.data_ptr()),
                                      None)
    assert rc == 0
    out = from_dev(dst, dt)
    cnt = d_cnt.cpu().numpy()
    for s in range(nseg):
        b, e = offs[s], offs[s + 1]
        ref, nlt, neq, ngt = orc.three_way_split(np.ascontiguousarray(a[b:e]), code, piv[s:s + 1])
        assert (cnt[2 * s], cnt[2 * s + 1]) == (nlt, ngt)
        # the <p and >p regions hold exactly the right multisets (order inside a region
        # is the kernel's own); compare sorted by the oracle's total order
        left = np.ascontiguousarray(out[b:b + nlt])
        right = np.ascontiguousarray(out[e - ngt:e])
        assert oracle_sort(orc, left, code).tobytes() == oracle_sort(orc, np.ascontiguousarray(ref[:nlt]), code).tobytes()
        assert oracle_sort(orc, right, code).tobytes() == oracle_sort(orc, np.ascontiguousarray(ref[nlt + neq:]), code).tobytes()


def test_small_sorter_every_size(T, orc):
    """Leaf kernel alone: one segment of every size 1..4096 (int32), then a sample of
    sizes for every other kind."""
    sizes = np.arange(1, 4097, dtype=np.int64)
    offs = np.zeros(len(sizes) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    a = int32_pattern("random", int(offs[-1]), seed=21)
    a[::5] = 7
    t = to_dev(a)
    d_offs = torch.from_numpy(offs).cuda()
    rc = T.lib().tsqs_debug_small_sort(ctypes.c_void_p(t.data_ptr()), int(offs[-1]), 4, 1,
                                       ctypes.c_void_p(d_offs.data_ptr()), len(sizes), None)
    assert rc == 0
    got = from_dev(t, np.int32)
    exp = a.copy()
    orc.tsqs_sort_segments(exp, offs.astype(np.uint64), 1, threads=4)
    assert got.tobytes() == exp.tobytes()
    for kind_name in ("u32", "f32", "i64", "u64", "f64"):
        code, dt, _ = KINDS[kind_name]
        sz = np.array([1, 2, 3, 17, 255, 256, 257, 1000, 2048, 4095, 4096], np.int64)
        of = np.zeros(len(sz) + 1, np.int64)
        of[1:] = np.cumsum(sz)
        x = random_keys(kind_name, int(of[-1]), seed=22)
        tx = to_dev(x)
        d_of = torch.from_numpy(of).cuda()
        assert T.lib().tsqs_debug_small_sort(ctypes.c_void_p(tx.data_ptr()), int(of[-1]), x.itemsize,
                                             code, ctypes.c_void_p(d_of.data_ptr()), len(sz), None) == 0
        ex = x.copy()
        orc.tsqs_sort_segments(ex, of.astype(np.uint64), code, threads=4)
        assert from_dev(tx, dt).tobytes() == ex.tobytes()


def test_segmented_matches_oracle(T, orc):
    offs, sizes, pat = batched_segments(600, seed=3, max_log2=16)
    x = batched_keys(offs, pat, seed=3)
    t = to_dev(x)
    d_offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    T.sort_segmented_(t, d_offs, kind=1)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    exp = x.copy()
    orc.tsqs_sort_segments(exp, offs, 1, threads=4)
    assert from_dev(t, np.int32).tobytes() == exp.tobytes()


def test_segmented_edge_cases(T, orc):
    sizes = np.array([0, 1, 0, 2, 4096, 4097, 0, 1, 100_000, 3], np.int64)
    offs = np.zeros(len(sizes) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    x = int32_pattern("many_equals", int(offs[-1]), seed=8)
    t = to_dev(x)
    T.sort_segmented_(t, torch.from_numpy(offs).cuda(), kind=1)
    torch.cuda.synchronize()
    exp = x.copy()
    orc.tsqs_sort_segments(exp, offs.astype(np.uint64), 1)
    assert from_dev(t, np.int32).tobytes() == exp.tobytes()


def test_argument_errors(T):
    L = T.lib()
    t = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    assert L.tsqs_sort(p, 16, 8, 1, None) == T.TSQS_EINVAL          # size mismatch
    assert L.tsqs_sort(p, 16, 4, 99, None) == T.TSQS_EINVAL         # unknown kind
    assert L.tsqs_sort(None, 16, 4, 1, None) == T.TSQS_EINVAL       # null base
    assert L.tsqs_sort(ctypes.c_void_p(t.data_ptr() + 2), 4, 4, 1, None) == T.TSQS_EINVAL
    assert L.tsqs_sort(None, 0, 4, 1, None) == T.TSQS_OK            # empty
    assert L.tsqs_sort(p, 1, 4, 1, None) == T.TSQS_OK


def test_bounded_wait_expires_to_etimeout(T):
    """A tile that never publishes its look-back word (injected on the host) makes the
    waits of its successors hit their poll limit; the sort must end with
    TSQS_ETIMEOUT instead of hanging, and the context must stay usable."""
    L = T.lib()
    a = int32_pattern("random", 1 << 20, seed=2)
    t = to_dev(a)
    L.tsqs_debug_set_spin_limit(2000)
    L.tsqs_debug_withhold_publish(1)
    try:
        T.sort_(t, kind=1)
        st = T.last_device_status()
    finally:
        L.tsqs_debug_withhold_publish(0)
        L.tsqs_debug_set_spin_limit(0)
    assert st == T.TSQS_ETIMEOUT
    t2 = to_dev(a)
    T.sort_(t2, kind=1)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    assert np.array_equal(t2.cpu().numpy(), np.sort(a))


def test_context_stats(T):
    ctx = T.Context()
    a = int32_pattern("random", 1 << 22, seed=3)
    t = to_dev(a)
    T.sort_(t, kind=1, ctx=ctx)
    st = ctx.stats()
    assert ctx.status() == 0
    assert st["leaf_sorted_keys"] + st["leaf_filled_keys"] + st["presorted_keys"] == len(a)
    assert st["levels"] >= 10 and st["level_keys"][0] == len(a)
    assert np.array_equal(t.cpu().numpy(), np.sort(a))
    ctx.close()


@pytest.mark.parametrize("offset_mode", [0, 1])
def test_offset_modes_match_oracle(T, orc, offset_mode):
    """Both ways of placing a tile's runs (per-segment atomic cursor, decoupled
    look-back) give the oracle's output."""
    plan = T.Plan()
    assert T.lib().tsqs_plan_default(1, 0, ctypes.byref(plan)) == 0
    plan.offset_mode = offset_mode
    ctx = T.Context(plan)
    for pattern in ("random", "many_equals", "organ_pipe"):
        a = int32_pattern(pattern, 2_000_003, seed=offset_mode + 1)
        t = to_dev(a)
        T.sort_(t, kind=1, ctx=ctx)
        assert ctx.status() == 0
        assert from_dev(t, np.int32).tobytes() == oracle_sort(orc, a, 1).tobytes()
    ctx.close()


# ------------------------------------------------------------------------------
# host-memory entry point: pinned arrays get the result straight from the kernels,
# pageable ones a copy after the sort; both at every 16-byte phase
# ------------------------------------------------------------------------------

@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("off", [0, 1, 3])
def test_host_sort_int32_matches_oracle(T, orc, pinned, off):
    n = 300_007
    a = int32_pattern("random", n + off + 2, seed=21 + off)
    exp = oracle_sort(orc, a[off:off + n], 1)
    h = torch.from_numpy(a.copy())
    if pinned:
        h = h.pin_memory()
    view = h[off:off + n]
    rc = T.lib().tsqs_sort_host(ctypes.c_void_p(view.data_ptr()), n, 4, 1, None)
    assert rc == 0
    got = h.numpy()
    assert got[off:off + n].tobytes() == exp.tobytes()
    assert got[:off].tobytes() == a[:off].tobytes()               # neighbours untouched
    assert got[off + n:].tobytes() == a[off + n:].tobytes()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_sort_records_matches_oracle(T, orc, pinned):
    n = 70_001
    r = records_u64(n, seed=33)
    exp = r.copy()
    orc.tsqs_sort(exp, 7)
    h = torch.from_numpy(r.view(np.int64).copy())
    if pinned:
        h = h.pin_memory()
    rc = T.lib().tsqs_sort_host(ctypes.c_void_p(h.data_ptr()), n, 16, 7, None)
    assert rc == 0
    assert h.numpy().view(np.uint64).reshape(n, 2).tobytes() == exp.tobytes()



# ------------------------------------------------------------------------------
# presortedness: root segments whose sample is in order are checked in full and, if
# they pass, finished as they stand or by one reversal; any defect falls back to the
# full sort.  Every case is compared with the oracle and with the statistics.
# ------------------------------------------------------------------------------

def _presort_inputs(n):
    i = np.arange(n, dtype=np.int64)
    asc = (i - n // 2).astype(np.int32)
    cases = {
        "sorted": (asc.copy(), n),
        "reversed": (asc[::-1].copy(), n),
        "stair_steps": ((i // 1024).astype(np.int32), n),
        "descending_runs": ((-(i // 777)).astype(np.int32), n),
        "all_equal": (np.full(n, 7, np.int32), n),
    }
    last = asc.copy(); last[-2], last[-1] = last[-1], last[-2]
    first = asc.copy(); first[0], first[1] = first[1], first[0]
    mid = asc[::-1].copy(); mid[n // 2] = mid[0] + 5
    cases["sorted_defect_at_end"] = (last, 0)
    cases["sorted_defect_at_start"] = (first, 0)
    cases["reversed_defect_in_middle"] = (mid, 0)
    cases["nearly_sorted"] = (int32_pattern("nearly_sorted", n, seed=4), 0)
    return cases


@pytest.mark.parametrize("case", ["sorted", "reversed", "stair_steps", "descending_runs", "all_equal",
                                  "sorted_defect_at_end", "sorted_defect_at_start",
                                  "reversed_defect_in_middle", "nearly_sorted"])
def test_presorted_inputs_match_oracle(T, orc, case):
    n = 1_000_003
    a, presorted = _presort_inputs(n)[case]
    ctx = T.Context()
    t = to_dev(a)
    T.sort_(t, kind=1, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert from_dev(t, np.int32).tobytes() == oracle_sort(orc, a, 1).tobytes()
    st = ctx.stats()
    assert st["presorted_keys"] == presorted
    assert st["leaf_sorted_keys"] + st["leaf_filled_keys"] + st["presorted_keys"] == n
    ctx.close()


def test_presorted_segments_mixed_with_others(T, orc):
    rng = np.random.default_rng(8)
    parts, offs, expect_pre = [], [0], 0
    for k in range(40):
        m = int(rng.integers(1, 60_000))
        kind = k % 5
        i = np.arange(m)
        if kind == 0:
            x = np.sort(rng.integers(-1000, 1000, m)).astype(np.int32)
        elif kind == 1:
            x = np.sort(rng.integers(-1000, 1000, m))[::-1].astype(np.int32)
        elif kind == 2:
            x = rng.integers(-2**31, 2**31 - 1, m).astype(np.int32)
        elif kind == 3:
            x = (i // 3).astype(np.int32)
            if m > 10:
                x[m // 2], x[m // 2 + 1] = x[m // 2 + 1] + 1, x[m // 2]
        else:
            x = np.zeros(m, np.int32)
        if kind in (0, 1, 4) and m > 4096:
            expect_pre += m
        parts.append(x)
        offs.append(offs[-1] + m)
    a = np.concatenate(parts)
    offs = np.array(offs, dtype=np.int64)
    ctx = T.Context()
    t = to_dev(a)
    T.sort_segmented_(t, torch.from_numpy(offs).cuda(), kind=1, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    exp = a.copy()
    orc.tsqs_sort_segments(exp, offs.astype(np.uint64), 1, threads=4)
    assert from_dev(t, np.int32).tobytes() == exp.tobytes()
    assert ctx.stats()["presorted_keys"] == expect_pre
    ctx.close()


def test_presorted_records_and_floats(T, orc):
    n = 200_001
    r = records_u64(n, seed=5)
    r = r[np.lexsort((r[:, 1], r[:, 0]))][::-1].copy()          # descending (key, payload)
    t = torch.from_numpy(r.view(np.int64).copy()).cuda()
    T.sort_(t, records=True)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    assert t.cpu().numpy().view(np.uint64).reshape(n, 2).tobytes() == oracle_sort(orc, r, 7).tobytes()
    f = floats_normal_specials(n, seed=6)
    f = f[np.argsort(total_order_key_f32(f), kind="stable")].copy()   # ascending totalOrder
    got = gpu_sort(T, f, 3)
    assert got.tobytes() == oracle_sort(orc, f, 3).tobytes()
    got = gpu_sort(T, f[::-1].copy(), 3)
    assert got.tobytes() == oracle_sort(orc, f, 3).tobytes()


@pytest.mark.parametrize("case", ["sorted", "reversed", "sorted_defect_at_end"])
def test_presorted_host_array(T, orc, case):
    n = 300_001
    a, _ = _presort_inputs(n)[case]
    exp = oracle_sort(orc, a, 1)
    h = torch.from_numpy(a.copy()).pin_memory()
    assert T.lib().tsqs_sort_host(ctypes.c_void_p(h.data_ptr()), n, 4, 1, None) == 0
    assert h.numpy().tobytes() == exp.tobytes()


def test_presorted_many_segments_checked_concurrently(T, orc):
    """Thousands of candidate segments checked by many blocks at once, with defects at
    random places: flags are cleared while other blocks are still checking."""
    rng = np.random.default_rng(19)
    parts, offs = [], [0]
    for k in range(6000):
        m = int(rng.integers(4097, 20_000))
        x = np.sort(rng.integers(-10**6, 10**6, m)).astype(np.int32)
        if k % 2:
            x = x[::-1].copy()
        if k % 3 == 0:
            j = int(rng.integers(0, m - 1))
            x[j], x[j + 1] = x[j + 1], x[j]
            if x[j] == x[j + 1]:
                x[j] += 1
        parts.append(x)
        offs.append(offs[-1] + m)
    a = np.concatenate(parts)
    offs = np.array(offs, dtype=np.int64)
    t = to_dev(a)
    T.sort_segmented_(t, torch.from_numpy(offs).cuda(), kind=1)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    exp = a.copy()
    orc.tsqs_sort_segments(exp, offs.astype(np.uint64), 1, threads=4)
    assert from_dev(t, np.int32).tobytes() == exp.tobytes()


def test_segmented_half_a_million_segments(T, orc):
    """Very many segments (most below 64 elements, a few above the on-chip threshold):
    the init pushes and the leaf queue are sized by the segment count."""
    rng = np.random.default_rng(77)
    nseg = 500_000
    sizes = rng.integers(0, 64, nseg).astype(np.int64)
    sizes[rng.integers(0, nseg, 40)] = rng.integers(4097, 300_000, 40)
    offs = np.zeros(nseg + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    x = int32_pattern("random", int(offs[-1]), seed=78)
    x[::9] = 5
    t = to_dev(x)
    T.sort_segmented_(t, torch.from_numpy(offs).cuda(), kind=1)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    exp = x.copy()
    orc.tsqs_sort_segments(exp, offs.astype(np.uint64), 1, threads=4)
    assert from_dev(t, np.int32).tobytes() == exp.tobytes()
