"""Seeded, bit-reproducible input generators (numpy, vectorised).

Random numbers come from SplitMix64 used as a counter-based generator: output i of
stream (seed, tag) is the SplitMix64 finaliser applied to x0 + (i + 1) * 0x9E3779B97F4A7C15,
which is exactly the i-th output of the published SplitMix64 generator started at state
x0 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", 2014).
x0 is derived from (seed, tag) with the same finaliser.

The seven orderings follow the paper's test inputs (Section VI: random, sorted,
reversed, organ pipes, many equals, stair steps, nearly sorted).  Records are 64-bit
keys with 64-bit payloads and some duplicated keys and records; floats are normal
draws with +-0, +-inf and NaNs of both signs mixed in.
"""
from __future__ import annotations

import numpy as np

PATTERNS = ("random", "sorted", "reversed", "organ_pipe", "many_equals", "stair_steps",
            "nearly_sorted")

_GOLD = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_state(seed: int, tag: int) -> np.uint64:
    with np.errstate(over="ignore"):
        x = np.array([(int(seed) * 0x2545F4914F6CDD1D + int(tag) * 0x632BE59BD9B4E019)
                      & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix(x)[0]


def splitmix64(x0: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 started at state x0."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(np.uint64(x0) + i * _GOLD)


def rand_u64(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    """count uniform uint64 values of stream (seed, tag)."""
    return splitmix64(int(_stream_state(seed, tag)), count, start)


def _unit(u: np.ndarray) -> np.ndarray:
    """uint64 -> float64 in [0, 1) from the top 53 bits."""
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ------------------------------------------------------------------------------
# int32 orderings (Section VI patterns)
# ------------------------------------------------------------------------------

def int32_pattern(name: str, n: int, seed: int = 1) -> np.ndarray:
    """The seven int32 test patterns.

    random        uniform over [-2^31, 2^31)
    sorted        a[i] = i
    reversed      a[i] = n - 1 - i
    organ_pipe    1, 2, ..., n/2, ..., 2, 1  (a[i] = i + 1 below n/2, n - i above)
    many_equals   uniform over [0, 16)
    stair_steps   runs of 1024 equal values, ascending: a[i] = i // 1024
    nearly_sorted a[i] = i, then n/200 disjoint random transpositions (1% of positions)
    """
    if n < 0:
        raise ValueError("n must be >= 0")
    i = np.arange(n, dtype=np.int64)
    if name == "random":
        return (rand_u64(seed, 1, n) >> np.uint64(32)).astype(np.uint32).view(np.int32)
    if name == "sorted":
        return i.astype(np.int32)
    if name == "reversed":
        return (n - 1 - i).astype(np.int32)
    if name == "organ_pipe":
        h = n // 2
        return np.where(i < h, i + 1, n - i).astype(np.int32)
    if name == "many_equals":
        return (rand_u64(seed, 2, n) >> np.uint64(60)).astype(np.int32)
    if name == "stair_steps":
        return (i // 1024).astype(np.int32)
    if name == "nearly_sorted":
        a = i.astype(np.int32)
        m = n // 200
        if m == 0 or n < 2:
            return a
        pos = (rand_u64(seed, 3, 2 * m) % np.uint64(n)).astype(np.int64)
        _, first = np.unique(pos, return_index=True)
        pos = pos[np.sort(first)]                       # distinct, in draw order
        k = len(pos) // 2
        p1, p2 = pos[:k], pos[k:2 * k]
        a[p1], a[p2] = a[p2].copy(), a[p1].copy()
        return a
    raise ValueError(f"unknown pattern {name!r}")


# ------------------------------------------------------------------------------
# 16-byte records and float32 with specials
# ------------------------------------------------------------------------------

def records_u64(n: int, seed: int = 1, dup_key_frac: float = 0.10,
                dup_rec_frac: float = 0.001) -> np.ndarray:
    """(n, 2) uint64 records (key, payload).  Keys and payloads uniform; a fraction
    dup_key_frac of records take the key of another uniformly chosen record, and a
    fraction dup_rec_frac take its payload too (exact duplicates)."""
    key = rand_u64(seed, 10, n)
    pay = rand_u64(seed, 11, n)
    u = _unit(rand_u64(seed, 12, n))
    src = (rand_u64(seed, 13, n) % np.uint64(max(n, 1))).astype(np.int64)
    out = np.empty((n, 2), dtype=np.uint64)
    out[:, 0] = np.where(u < dup_key_frac, key[src], key)
    out[:, 1] = np.where(u < dup_rec_frac, pay[src], pay)
    return out


def floats_normal_specials(n: int, seed: int = 1, special_frac: float = 0.001) -> np.ndarray:
    """float32 ~ N(0, 1) by Box-Muller, then special_frac of positions replaced in equal
    shares by +0.0, -0.0, +inf, -inf, +NaN, -NaN; NaNs get random nonzero payloads with
    the quiet bit random (quiet and signalling NaNs both occur)."""
    u1 = 1.0 - _unit(rand_u64(seed, 20, n))          # (0, 1]
    u2 = _unit(rand_u64(seed, 21, n))
    z = (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).astype(np.float32)
    bits = z.view(np.uint32).copy()
    sel = _unit(rand_u64(seed, 22, n)) < special_frac
    cls = (rand_u64(seed, 23, n) % np.uint64(6)).astype(np.int64)
    mant = (rand_u64(seed, 24, n) >> np.uint64(41)).astype(np.uint32) & np.uint32(0x7FFFFF)
    mant = np.where(mant == 0, np.uint32(1), mant)
    table = np.array([0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7F800000, 0xFF800000],
                     dtype=np.uint32)
    sp = table[cls] | np.where(cls >= 4, mant, np.uint32(0))
    bits = np.where(sel, sp, bits).astype(np.uint32)
    return bits.view(np.float32)


# ------------------------------------------------------------------------------
# batched and serving workloads
# ------------------------------------------------------------------------------

def batched_segments(nseg: int, seed: int = 1, max_log2: int = 20):
    """Segment sizes floor(2^(max_log2 * U)) clamped to [1, 2^max_log2] and one pattern
    index per segment.  Returns (offsets[nseg+1] uint64, sizes int64, pattern idx int64)."""
    u = _unit(rand_u64(seed, 30, nseg))
    sizes = np.floor(np.exp2(max_log2 * u)).astype(np.int64)
    sizes = np.clip(sizes, 1, 1 << max_log2)
    pat = (rand_u64(seed, 31, nseg) % np.uint64(len(PATTERNS))).astype(np.int64)
    offs = np.zeros(nseg + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(sizes).astype(np.uint64)
    return offs, sizes, pat


def batched_keys(offs: np.ndarray, pat: np.ndarray, seed: int = 1) -> np.ndarray:
    """The int32 keys of a batched workload: segment s holds pattern pat[s] of its size,
    generated with seed (seed * 1000003 + s)."""
    total = int(offs[-1])
    out = np.empty(total, dtype=np.int32)
    for s in range(len(pat)):
        lo, hi = int(offs[s]), int(offs[s + 1])
        out[lo:hi] = int32_pattern(PATTERNS[int(pat[s])], hi - lo, seed * 1000003 + s)
    return out


def serving_requests(nreq: int, seed: int = 1, lo_log2: int = 10, hi_log2: int = 24,
                     rec_frac: float = 0.30):
    """Request mix: sizes floor(2^(lo + (hi - lo) U)), key kind 'rec' with probability
    rec_frac (else 'i32'), a pattern index, and unit-rate exponential inter-arrival gaps
    (scale them by 1/lambda).  Returns a dict of numpy arrays."""
    u = _unit(rand_u64(seed, 40, nreq))
    sizes = np.floor(np.exp2(lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)
    is_rec = _unit(rand_u64(seed, 41, nreq)) < rec_frac
    pat = (rand_u64(seed, 42, nreq) % np.uint64(len(PATTERNS))).astype(np.int64)
    gaps = -np.log(1.0 - _unit(rand_u64(seed, 43, nreq)))
    return {"sizes": sizes, "is_rec": is_rec, "pattern": pat, "gaps": gaps}


# ------------------------------------------------------------------------------
# sort keys for checking results against a library sort
# ------------------------------------------------------------------------------

def total_order_key_f32(x: np.ndarray) -> np.ndarray:
    """int64 key whose numeric order is IEEE totalOrder on float32 bit patterns:
    negatives by decreasing magnitude below positives by increasing magnitude."""
    b = np.ascontiguousarray(x).view(np.uint32).astype(np.int64)
    mag = b & 0x7FFFFFFF
    return np.where(b >> 31, -mag - 1, mag)


def total_order_key_f64(x: np.ndarray):
    """(hi, lo) pair of arrays for float64 totalOrder, for np.lexsort((lo, hi))."""
    b = np.ascontiguousarray(x).view(np.uint64)
    neg = (b >> np.uint64(63)).astype(bool)
    mag = b & np.uint64(0x7FFFFFFFFFFFFFFF)
    # order: negatives (larger magnitude first) then positives (smaller first)
    hi = neg.astype(np.int8) * -1 + 1                    # 0 for negative, 1 for positive
    lo = np.where(neg, np.uint64(0x7FFFFFFFFFFFFFFF) - mag, mag)
    return hi, lo
