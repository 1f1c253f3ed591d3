"""The benchmark configurations at full size, through the same entry points the bench
times (tsqs_sort / tsqs_sort_segmented on the default context, one graph launch).

At these sizes the output is checked three ways, none of which uses the CUDA path:
  - element by element against the CPU oracle, for every configuration (the sorted
    output is unique, so the comparison is byte for byte; the oracle sorts run on the
    host's cores in parallel while the GPU works);
  - at sampled positions k, one by one from the definition of the sorted order: the
    element at k has fewer than k + 1 input elements below it and more than k at or
    below it (counted on the CPU over the input);
  - by properties that hold at any size: adjacent elements in order, and the sorted
    multiset equal to that of the input (a library sort of the input on the device).
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from workloads import PATTERNS, int32_pattern, records_u64, floats_normal_specials, total_order_key_f32
from workloads.patterns import batched_segments, batched_keys

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


_POOL = ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) - 1)))


def _oracle_async(orc, a: np.ndarray, kind: int):
    """Starts the oracle on a private copy of a (the oracle releases the GIL); returns a
    future of the sorted bytes."""
    def run():
        exp = a.copy()
        orc.tsqs_sort(exp, kind)
        return exp.tobytes()
    return _POOL.submit(run)


def _sampled_ranks_ok(order_key_in: np.ndarray, order_key_out_at, ks) -> None:
    """order_key_in: totally ordered integer image of the input (numpy); for each k the
    output element's image v must satisfy #(in < v) <= k < #(in <= v)."""
    for k in ks:
        v = order_key_out_at(k)
        lt = int(np.count_nonzero(order_key_in < v))
        le = int(np.count_nonzero(order_key_in <= v))
        assert lt <= k < le, f"rank check failed at {k}"


def _ks(n, seed, m=40):
    rng = np.random.default_rng(seed)
    return sorted(set([0, 1, n // 2, n - 2, n - 1] + [int(x) for x in rng.integers(0, n, m)]))


def test_full_2e27_uniform_int32_matches_oracle(T, orc):
    n = 1 << 27
    a = int32_pattern("random", n, seed=1)
    t = torch.from_numpy(a).cuda()
    T.sort_(t)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    got = t.cpu().numpy()
    exp = a.copy()
    orc.tsqs_sort(exp, 1)
    assert got.tobytes() == exp.tobytes()
    _sampled_ranks_ok(a, lambda k: got[k], _ks(n, 1))


@pytest.mark.parametrize("pattern", PATTERNS[1:])
def test_full_2e27_patterns(T, orc, pattern):
    n = 1 << 27
    a = int32_pattern(pattern, n, seed=1)
    fut = _oracle_async(orc, a, orc.KIND_I32)
    src = torch.from_numpy(a).cuda()
    t = src.clone()
    T.sort_(t)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    assert bool((t[1:] >= t[:-1]).all().item())
    assert torch.equal(t, torch.sort(src)[0])
    got = t.cpu().numpy()
    _sampled_ranks_ok(a, lambda k: got[k], _ks(n, 2, m=12))
    assert got.tobytes() == fut.result()


def test_full_2e26_records(T, orc):
    n = 1 << 26
    r = records_u64(n, seed=1)
    fut = _oracle_async(orc, r, orc.KIND_REC)
    t = torch.from_numpy(r.view(np.int64).copy()).cuda()
    T.sort_(t, records=True)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    got = t.cpu().numpy().view(np.uint64).reshape(n, 2)
    # in order by (key, payload)
    k, p = got[:, 0], got[:, 1]
    assert bool(np.all((k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (p[1:] >= p[:-1]))))
    # same multiset: identical after a lexicographic library sort of the input
    idx = np.lexsort((r[:, 1], r[:, 0]))
    assert got.tobytes() == r[idx].tobytes()
    assert got.tobytes() == fut.result()


def test_full_2e26_floats_total_order(T, orc):
    n = 1 << 26
    f = floats_normal_specials(n, seed=1)
    fut = _oracle_async(orc, f, orc.KIND_F32)
    t = torch.from_numpy(f.copy()).cuda()
    T.sort_(t, kind=3)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    got = t.cpu().numpy()
    kin = total_order_key_f32(f)
    kout = total_order_key_f32(got)
    assert bool(np.all(kout[1:] >= kout[:-1]))
    assert np.array_equal(np.sort(kin), kout)
    _sampled_ranks_ok(kin, lambda k: kout[k], _ks(n, 3))
    assert got.tobytes() == fut.result()


def test_full_batched_20000_segments(T, orc):
    nseg = 20_000
    offs, sizes, pat = batched_segments(nseg, seed=1)
    x = batched_keys(offs, pat, seed=1)
    exp = x.copy()

    def oracle_all():                  # every segment, on all host cores but one
        orc.tsqs_sort_segments(exp, offs, orc.KIND_I32, threads=max(1, (os.cpu_count() or 2) - 1))
    fut = _POOL.submit(oracle_all)
    src = torch.from_numpy(x).cuda()
    d_offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    t = src.clone()
    T.sort_segmented_(t, d_offs, kind=1)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    # every segment in order, and each segment the same multiset: (segment, key) pairs
    # of output and input agree after a library sort
    seg = torch.repeat_interleave(torch.arange(nseg, device="cuda", dtype=torch.int64),
                                  torch.from_numpy(np.diff(offs).astype(np.int64)).cuda())
    comb_out = (seg << 32) | (t.to(torch.int64) + 2**31)
    assert bool((comb_out[1:] >= comb_out[:-1]).all().item())
    comb_in = (seg << 32) | (src.to(torch.int64) + 2**31)
    assert torch.equal(torch.sort(comb_in)[0], comb_out)
    del comb_in, comb_out, seg
    # all 20,000 segments against the oracle, element by element
    got = t.cpu().numpy()
    fut.result()
    if got.tobytes() != exp.tobytes():
        bad = [s for s in range(nseg)
               if got[offs[s]:offs[s + 1]].tobytes() != exp[offs[s]:offs[s + 1]].tobytes()]
        raise AssertionError(f"{len(bad)} segments differ from the oracle, first {bad[:5]}")


@pytest.mark.parametrize("mode", [0, 1])
def test_largest_segment_2e31_minus_1(T, mode):
    """The largest segment the boundary accepts (2^31 - 1 int32): tile ids, per-tile
    counts, per-segment cursors and look-back words all run at their widest.  Checked on
    the device by properties (in order; equal to a library sort of the input)."""
    import ctypes
    n = (1 << 31) - 1
    free, _ = torch.cuda.mem_get_info()
    if free < 48 * (1 << 30):
        pytest.skip("needs about 48 GB of device memory")
    g = torch.Generator(device="cuda")
    g.manual_seed(31 + mode)
    src = torch.randint(-2**31, 2**31, (n,), dtype=torch.int64, device="cuda", generator=g).to(torch.int32)
    plan = T.Plan()
    T.lib().tsqs_plan_default(T.TSQS_I32, n, ctypes.byref(plan))
    plan.offset_mode = mode
    ctx = T.Context(plan)
    t = src.clone()
    T.sort_(t, kind=T.TSQS_I32, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert bool((t[1:] >= t[:-1]).all().item())
    ref = torch.sort(src)[0]
    del src
    assert torch.equal(t, ref)
    ctx.close()
