"""The oracle's sorted result against library sorts on the workload patterns.

The sorted output under a total order is unique, so numpy's sort (on integers
directly, on floats through the IEEE totalOrder key, on records through lexsort)
pins every output element.
"""
import numpy as np
import pytest

from workloads import (PATTERNS, int32_pattern, records_u64, floats_normal_specials,
                       total_order_key_f32, total_order_key_f64, rand_u64)


@pytest.mark.parametrize("pattern", PATTERNS)
@pytest.mark.parametrize("n", [1000, 100_000])
def test_int32_patterns(orc, pattern, n):
    x = int32_pattern(pattern, n, seed=3)
    a = x.copy()
    st = orc.tsqs_sort(a, orc.KIND_I32)
    np.testing.assert_array_equal(a, np.sort(x))
    assert st["stages"] > 0


def test_c1_one_million_uniform(orc):
    x = int32_pattern("random", 1_000_000, seed=1)
    a = x.copy()
    orc.tsqs_sort(a, orc.KIND_I32)
    np.testing.assert_array_equal(a, np.sort(x))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 16, 17, 69, 70, 799, 800, 40_000, 65_537])
def test_tier_boundaries(orc, n):
    """Sizes at each pivot tier boundary (Section III.H) and the insertion threshold."""
    for seed in (1, 2):
        x = int32_pattern("random", n, seed=seed)
        a = x.copy()
        orc.tsqs_sort(a, orc.KIND_I32)
        np.testing.assert_array_equal(a, np.sort(x))


def test_records(orc):
    r = records_u64(50_000, seed=4)
    a = r.copy()
    orc.tsqs_sort(a, orc.KIND_REC)
    order = np.lexsort((r[:, 1], r[:, 0]))
    np.testing.assert_array_equal(a, r[order])


def test_floats_total_order(orc):
    x = floats_normal_specials(60_000, seed=5, special_frac=0.05)
    a = x.copy()
    orc.tsqs_sort(a, orc.KIND_F32)
    expect = x[np.argsort(total_order_key_f32(x), kind="stable")]
    assert a.view(np.uint32).tolist() == expect.view(np.uint32).tolist()


def test_float64_total_order(orc):
    bits = rand_u64(6, 1, 40_000)
    # sprinkle specials: +-0, +-inf, NaNs with payloads
    bits[::97] = np.uint64(0x8000000000000000)
    bits[::89] = np.uint64(0)
    bits[::83] = np.uint64(0x7FF0000000000000)
    bits[::79] = np.uint64(0xFFF0000000000000)
    x = bits.view(np.float64)
    a = x.copy()
    orc.tsqs_sort(a, orc.KIND_F64)
    hi, lo = total_order_key_f64(x)
    expect = x[np.lexsort((lo, hi))]
    assert a.view(np.uint64).tolist() == expect.view(np.uint64).tolist()


@pytest.mark.parametrize("kind,dtype", [(2, np.uint32), (4, np.int64), (5, np.uint64)])
def test_other_integer_kinds(orc, kind, dtype):
    bits = rand_u64(7, kind, 30_000)
    x = bits.astype(dtype) if np.dtype(dtype).itemsize == 8 else (bits >> np.uint64(32)).astype(dtype)
    x[::10] = x[5]                                  # duplicates
    a = x.copy()
    orc.tsqs_sort(a, kind)
    np.testing.assert_array_equal(a, np.sort(x))


def test_segments_threads(orc):
    from workloads.patterns import batched_segments, batched_keys
    offs, sizes, pat = batched_segments(300, seed=2, max_log2=12)
    x = batched_keys(offs, pat, seed=2)
    a = x.copy()
    orc.tsqs_sort_segments(a, offs, orc.KIND_I32, threads=4)
    for s in range(300):
        lo, hi = int(offs[s]), int(offs[s + 1])
        np.testing.assert_array_equal(a[lo:hi], np.sort(x[lo:hi]))


def test_three_way_split_definition(orc):
    x = int32_pattern("many_equals", 1000, seed=8)
    out, lt, eq, gt = orc.three_way_split(x, orc.KIND_I32, 7)
    assert lt == (x < 7).sum() and eq == (x == 7).sum() and gt == (x > 7).sum()
    np.testing.assert_array_equal(out[:lt], x[x < 7])
    assert (out[lt:lt + eq] == 7).all()
    np.testing.assert_array_equal(out[lt + eq:], x[x > 7])


def test_lower_median(orc):
    rng = np.random.default_rng(1)
    for s in (1, 2, 3, 15, 31, 32, 63):
        k = rng.integers(-50, 50, s).astype(np.int32)
        m = orc.lower_median(k, orc.KIND_I32)
        assert m[0] == np.sort(k)[(s - 1) // 2]
