"""Pins of the oracle's large-element path (late swapping, Section VIII.H).

The definition: elements keep their bytes and are ordered by the key at key_offset
under the kind's total order, equal keys in their original order.  numpy's stable
argsort of an order-preserving integer image of the key is that definition written
with a library routine, so every case here is compared with it byte for byte.  The
move count is pinned by the structure of the permutation: every element not already
in place moves once, and each cycle adds one move through the temporary.
"""
import itertools

import numpy as np
import pytest

from workloads import rand_u64


def _order_key(keys: np.ndarray) -> np.ndarray:
    """Integer image of the keys whose numeric order is the kind's total order."""
    if keys.dtype == np.float32:
        b = keys.view(np.uint32).astype(np.int64)
        mag = b & 0x7FFFFFFF
        return np.where(b >> 31, -mag - 1, mag)
    if keys.dtype == np.float64:
        b = keys.view(np.uint64)
        mag = (b & np.uint64(0x7FFFFFFFFFFFFFFF)).astype(object)
        neg = (b >> np.uint64(63)).astype(bool)
        return np.array([-m - 1 if s else m for m, s in zip(mag, neg)], dtype=object)
    return keys.astype(object) if keys.dtype == np.uint64 else keys.astype(np.int64)


def _expected(raw: np.ndarray, n: int, es: int, off: int, dt) -> np.ndarray:
    el = raw.reshape(n, es)
    keys = np.ascontiguousarray(el[:, off:off + np.dtype(dt).itemsize]).view(dt).ravel()
    k = _order_key(keys)
    perm = sorted(range(n), key=lambda i: (k[i], i))          # stable: ties by position
    return el[perm].ravel()


def _cycle_counts(raw: np.ndarray, exp: np.ndarray, n: int, es: int):
    """(elements not in place, cycles) of the permutation the sort applies; the
    payload word after the key carries the original index in these inputs."""
    idx = exp.reshape(n, es)[:, -4:].copy().view(np.uint32).ravel().astype(np.int64)
    seen = np.zeros(n, bool)
    moved = cycles = 0
    for i in range(n):
        if seen[i] or idx[i] == i:
            seen[i] = True
            continue
        cycles += 1
        j = i
        while not seen[j]:
            seen[j] = True
            moved += 1
            j = idx[j]
    return moved, cycles


KEY_TYPES = {1: np.int32, 2: np.uint32, 3: np.float32, 4: np.int64, 5: np.uint64, 6: np.float64}


def _make(n, es, off, kind, seed, distinct=2**40):
    dt = KEY_TYPES[kind]
    raw = np.frombuffer(rand_u64(seed, 700, (n * es + 7) // 8).tobytes(), dtype=np.uint8)[:n * es].copy()
    el = raw.reshape(n, es)
    bits = rand_u64(seed, 701, n) % np.uint64(distinct)
    if np.dtype(dt).itemsize == 4:
        keys = (bits & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(dt).copy()
    else:
        keys = bits.view(dt).copy()
    if kind in (3, 6) and n > 12:
        sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan], dtype=dt)
        keys[3:9] = sp
    el[:, off:off + np.dtype(dt).itemsize] = keys.view(np.uint8).reshape(n, -1)
    el[:, -4:] = np.arange(n, dtype=np.uint32).view(np.uint8).reshape(n, 4)   # original index
    return raw


def test_wide_exhaustive_weak_orderings(orc):
    """Every weak ordering of 6 int32 keys in 16-byte elements lands in stable order."""
    n, es, off = 6, 16, 4
    for ranks in itertools.product(range(n), repeat=n):
        if sorted(set(ranks)) != list(range(len(set(ranks)))):
            continue                                              # not a weak ordering
        raw = np.zeros((n, es), np.uint8)
        raw[:, off:off + 4] = (np.array(ranks, np.int32) * 7 - 20).view(np.uint8).reshape(n, 4)
        raw[:, -4:] = np.arange(n, dtype=np.uint32).view(np.uint8).reshape(n, 4)
        raw = raw.ravel()
        exp = _expected(raw, n, es, off, np.int32)
        got = raw.copy()
        orc.wide_sort(got, es, off, 1)
        assert got.tobytes() == exp.tobytes()


@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("es,off", [(8, 0), (12, 4), (24, 8), (56, 16), (320, 256)])
def test_wide_matches_stable_sort(orc, kind, es, off):
    ks = np.dtype(KEY_TYPES[kind]).itemsize
    if off + ks > es - 4 or off % ks:
        pytest.skip("key does not fit before the index word")
    n = 3001
    for distinct in (2**40, 17):                                  # unique-ish and many equal keys
        raw = _make(n, es, off, kind, seed=es * 10 + kind, distinct=distinct)
        exp = _expected(raw, n, es, off, KEY_TYPES[kind])
        got = raw.copy()
        st = orc.wide_sort(got, es, off, kind)
        assert got.tobytes() == exp.tobytes()
        moved, cycles = _cycle_counts(raw, exp, n, es)
        assert st["cycles"] == cycles
        assert st["moves"] == moved + cycles


def test_wide_rejects_bad_arguments(orc):
    raw = np.zeros(64, np.uint8)
    with pytest.raises(RuntimeError):
        orc.wide_sort(raw, 8, 4, 4)          # 8-byte key does not fit at offset 4
    with pytest.raises(RuntimeError):
        orc.wide_sort(raw, 16, 0, 7)         # records are not a key kind here
