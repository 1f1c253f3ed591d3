"""The seeded generators: SplitMix64 against its published definition, and the
shapes and statistics of each workload pattern."""
import numpy as np
import pytest

from workloads import (PATTERNS, splitmix64, int32_pattern, records_u64,
                       floats_normal_specials, batched_segments, serving_requests)
from workloads.patterns import batched_keys

MASK = (1 << 64) - 1


def _splitmix_ref(x, count):
    """SplitMix64 as published: x += golden gamma, then the two xor-shift-multiply
    rounds and a final xor-shift, in plain Python integers."""
    out = []
    for _ in range(count):
        x = (x + 0x9E3779B97F4A7C15) & MASK
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def test_splitmix_first_output_seed0():
    # the first output of SplitMix64 started from state 0
    assert int(splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("x0", [0, 1, 1234567, 0xDEADBEEFCAFEF00D])
def test_splitmix_matches_reference(x0):
    assert [int(v) for v in splitmix64(x0, 50)] == _splitmix_ref(x0, 50)
    # counter-based: any window equals the sequential stream
    assert [int(v) for v in splitmix64(x0, 5, start=17)] == _splitmix_ref(x0, 22)[17:]


@pytest.mark.parametrize("pattern", PATTERNS)
def test_patterns_shape_and_determinism(pattern):
    n = 1 << 16
    a = int32_pattern(pattern, n, seed=3)
    b = int32_pattern(pattern, n, seed=3)
    assert a.dtype == np.int32 and a.shape == (n,)
    np.testing.assert_array_equal(a, b)


def test_pattern_definitions():
    n = 1 << 14
    i = np.arange(n)
    np.testing.assert_array_equal(int32_pattern("sorted", n), i)
    np.testing.assert_array_equal(int32_pattern("reversed", n), n - 1 - i)
    op = int32_pattern("organ_pipe", n)
    assert op[0] == 1 and op[n // 2 - 1] == n // 2 and op[n // 2] == n // 2 and op[-1] == 1
    assert int32_pattern("many_equals", n).max() < 16 and int32_pattern("many_equals", n).min() >= 0
    st = int32_pattern("stair_steps", n)
    assert (np.bincount(st) == 1024).all()
    ns = int32_pattern("nearly_sorted", n)
    moved = (ns != i).sum()
    assert 0 < moved <= n // 100 and np.array_equal(np.sort(ns), i)
    r = int32_pattern("random", 1 << 20)
    assert abs(r.astype(np.float64).mean()) < 2 ** 31 * 0.01


def test_records_and_floats():
    r = records_u64(1 << 16, seed=2)
    assert r.shape == (1 << 16, 2) and r.dtype == np.uint64
    dup_keys = len(r) - len(np.unique(r[:, 0]))
    assert 0.05 * len(r) < dup_keys < 0.15 * len(r)
    f = floats_normal_specials(1 << 18, seed=2, special_frac=0.01)
    b = f.view(np.uint32)
    nan = ((b & 0x7F800000) == 0x7F800000) & ((b & 0x7FFFFF) != 0)
    assert nan.sum() > 0 and (b == 0x80000000).sum() > 0 and (b == 0).sum() > 0
    assert ((b & 0x7FFFFF)[nan] & 0x400000).min() == 0      # some signalling NaNs
    assert ((b & 0x7FFFFF)[nan] & 0x400000).max() > 0       # some quiet NaNs
    assert abs(np.nanstd(f[np.isfinite(f)]) - 1) < 0.02


def test_batched_and_serving_mix():
    offs, sizes, pat = batched_segments(20_000, seed=1)
    assert len(offs) == 20_001 and sizes.min() >= 1 and sizes.max() <= 1 << 20
    assert int(offs[-1]) == int(sizes.sum())
    x = batched_keys(offs[:51], pat[:50], seed=1)
    assert len(x) == int(offs[50])
    req = serving_requests(5000, seed=1)
    assert req["sizes"].min() >= 1 << 10 and req["sizes"].max() <= 1 << 24
    assert 0.25 < req["is_rec"].mean() < 0.35
