"""Counter pins of the CPU oracle: the comparison and copy counts it reports are fixed
here by definitions and by the paper's closed forms, not by the oracle itself.

Exact, by definition (every input checked, so a single miscounted copy fails):
* the copy-based insertion sort of Section IV: an element that is smaller than the
  largest element of its sorted prefix costs one copy out, one copy per larger prefix
  element (the shifts) and one copy back; its comparisons are the first test against
  the prefix maximum, one per shift after the first, and a final failing test unless it
  reaches the front;
* the pivot samples of Section III.H: a median of three moves its elements by copies
  through one scratch element, so sorting three distinct values costs k + 1 copies per
  cycle of length k >= 2 of the sorting permutation; the median of five (and the
  fifteenther's median of the five group medians) is an insertion sort over the sample
  positions, with the insertion-sort counts above.

Whole sorts against Section V.A, 200 seeded random permutations of distinct int32 keys
at n = 10^4, 10^5 and 10^6, uniformly random pivot and no insertion sort:
* comparisons of Triple State and of the textbook Hoare quicksort against eq. (3);
* the Hoare exchanges against eq. (4); the two-way juggling partition of Section II
  (the model behind eqs. (5)-(8)) against eq. (8);
* the n ln n coefficients, read as slopes of count / n against ln n between the sizes:
  2 for comparisons (eq. (3)), 1/3 for exchanges (eq. (4)), 2/9 for the juggling
  partition's virtual swaps (eq. (9));
* the "about 2/3" of the abstract: Triple State's virtual swaps (copies / 3) over the
  Hoare exchanges, as the ratio of the two n ln n coefficients, in [0.60, 0.80];
* Triple State's copies less five per stage (the copies into and out of p and temp and
  the refill of the pivot's slot) against three times eq. (8): within 5% for n >= 10^5,
  within 8% at n = 10^4, where the linear terms, which the model gets only roughly,
  weigh more.
The paper's full configuration (tiered pivots, insertion sort below 17 elements) is
reported beside them.
"""
import ctypes
import itertools
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle.oracle import _Cfg, _Stats

I32 = 1


def bind(L):
    """Sets the argument types of the oracle entry points these pins call on a loaded
    oracle library (the committed one, or a planted mutant)."""
    vp, sz, i, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64
    ps, pc = ctypes.POINTER(_Stats), ctypes.POINTER(_Cfg)
    L.orc_tsqs_sort.argtypes = [vp, sz, i, pc, ps]
    L.orc_tsqs_sort_rows.argtypes = [vp, sz, sz, i, pc, ps]
    L.orc_classical_sort.argtypes = [vp, sz, i, u64, ps]
    L.orc_juggle_sort.argtypes = [vp, sz, i, u64, ps]
    L.orc_choose_pivot.argtypes = [vp, sz, i, pc, ps]
    L.orc_choose_pivot.restype = ctypes.c_longlong
    return L


def _cfg(ins_threshold=16, pivot_policy=0, random_samples=1, seed=1):
    return _Cfg(ins_threshold, pivot_policy, random_samples, 70, 800, 40000, seed)


# ----------------------------------------------------------------------------------
# Exact pins by definition
# ----------------------------------------------------------------------------------

def insertion_counts(rows: np.ndarray) -> tuple[int, int]:
    """Comparisons and copies of a copy-based insertion sort of every row (Section IV),
    from the inversion structure of the input."""
    rows = np.atleast_2d(rows)
    cm = mv = 0
    for k in range(1, rows.shape[1]):
        d = (rows[:, :k] > rows[:, k:k + 1]).sum(axis=1)          # larger prefix elements
        moved = d > 0
        cm += rows.shape[0]                                        # test against prefix max
        cm += int(((d - 1) * moved).sum()) + int((moved & (d < k)).sum())
        mv += int(((d + 2) * moved).sum())
    return cm, mv


def cycle_copies(vals) -> int:
    """Copies needed to sort distinct values in place through one scratch element:
    k + 1 for every cycle of length k >= 2 of the sorting permutation."""
    dest = np.argsort(np.argsort(np.asarray(vals)))                # final slot of each value
    seen, total = set(), 0
    for s in range(len(vals)):
        if s in seen:
            continue
        k, j = 0, s
        while j not in seen:
            seen.add(j)
            j = int(dest[j])
            k += 1
        if k >= 2:
            total += k + 1
    return total


def insertion_sort_counts_fail(L) -> str | None:
    """None if the oracle's insertion sort counts match the definition on every input."""
    cases = []
    for n in range(2, 8):                                          # every permutation
        cases.append(np.array(list(itertools.permutations(range(n))), dtype=np.int32))
    rng = np.random.default_rng(21)
    for n in (8, 11, 16):
        cases.append(np.argsort(rng.random((400, n)), axis=1).astype(np.int32))
        cases.append(rng.integers(0, 3, (400, n)).astype(np.int32))  # with equal keys
    for rows in cases:
        a = np.ascontiguousarray(rows.copy())
        st = _Stats()
        cfg = _cfg(ins_threshold=16)
        L.orc_tsqs_sort_rows(a.ctypes.data, a.shape[0], a.shape[1], I32, ctypes.byref(cfg),
                             ctypes.byref(st))
        if not np.array_equal(a, np.sort(rows, axis=1)) or st.stages != 0:
            return f"n={rows.shape[1]}: not an insertion sort"
        cm, mv = insertion_counts(rows)
        if (st.cmps, st.moves) != (cm, mv):
            return f"n={rows.shape[1]}: counts {(st.cmps, st.moves)} != definition {(cm, mv)}"
    return None


def _pivot_positions(n: int) -> list[list[int]]:
    """Sample groups of the tier for a part of n elements with the V.C shift off, in
    the order the tier sorts them (Section III.H; readings 7 and 8 of the positions)."""
    b, mid = n - 1, (n - 1) // 2
    if n < 70:
        return [[0, mid, b]]
    if n < 800:
        g = n // 4
        return [[0, g, mid, b - g, b]]
    if n < 40000:
        q = [k * b // 8 for k in range(9)]
        return [q[0:3], q[3:6], q[6:9], [q[1], q[4], q[7]]]
    q = [k * b // 14 for k in range(15)]
    return [q[3 * g:3 * g + 3] for g in range(5)] + [[q[1], q[4], q[7], q[10], q[13]]]


def pivot_counts_fail(L) -> str | None:
    """None if pivot selection sorts every sample group in place with the copies the
    definition fixes (distinct keys), and returns mid."""
    rng = np.random.default_rng(22)
    for n in (3, 4, 5, 17, 69, 70, 101, 799, 800, 4097, 39999, 40000, 65537):
        for _ in range(60):
            x = rng.permutation(n).astype(np.int32)
            a = x.copy()
            st = _Stats()
            cfg = _cfg(random_samples=0)
            pi = L.orc_choose_pivot(a.ctypes.data, n, I32, ctypes.byref(cfg), ctypes.byref(st))
            if pi != (n - 1) // 2:
                return f"n={n}: pivot index {pi}"
            ref = x.copy()
            mv = 0
            cm_lo = cm_hi = 0
            for grp in _pivot_positions(n):
                v = ref[grp].copy()
                if len(grp) == 3:
                    mv += cycle_copies(v)
                    cm_lo, cm_hi = cm_lo + 2, cm_hi + 3
                else:
                    c, m = insertion_counts(v[None, :])
                    mv += m
                    cm_lo, cm_hi = cm_lo + c, cm_hi + c
                ref[grp] = np.sort(v)
            if not np.array_equal(a, ref):
                return f"n={n}: samples not sorted in place"
            if st.moves != mv:
                return f"n={n}: {st.moves} copies, definition {mv}"
            if not cm_lo <= st.cmps <= cm_hi:
                return f"n={n}: {st.cmps} comparisons outside [{cm_lo}, {cm_hi}]"
    return None


def test_insertion_sort_counts_by_definition(orc):
    assert insertion_sort_counts_fail(bind(orc.lib())) is None


def test_pivot_selection_counts_by_definition(orc):
    assert pivot_counts_fail(bind(orc.lib())) is None


def test_cycle_copies_examples():
    assert cycle_copies([1, 2, 3]) == 0
    assert cycle_copies([2, 1, 3]) == 3                           # one transposition
    assert cycle_copies([2, 3, 1]) == 4                           # one 3-cycle
    assert cycle_copies([2, 1, 4, 3]) == 6


# ----------------------------------------------------------------------------------
# Whole sorts against the closed forms of Section V.A
# ----------------------------------------------------------------------------------

def _H(n):
    return math.fsum(1.0 / k for k in range(1, n + 1))


def eq3(n):
    return 2 * n * math.log(n) - 2.8456 * n


def eq4(n):
    return 0.33 * n * math.log(n) - 0.58 * n


def eq8(n):
    return 2 / 9 * (n + 1) * _H(n) - (n + 1) / 6


def whole_sort_means(L, n: int, reps: int, full: bool = True, threads: int = 8) -> dict:
    """Mean counters over `reps` seeded permutations of 0..n-1: Triple State with a
    uniformly random pivot and no insertion sort ("ts"), the Hoare baseline ("hoare"),
    the juggling partition ("juggle") and, if `full`, Triple State in the paper's
    configuration ("full")."""
    def one(r):
        x = np.random.default_rng([n, r]).permutation(n).astype(np.int32)
        out = {}
        for name, call in (
                ("ts", lambda a, st: L.orc_tsqs_sort(a.ctypes.data, n, I32, ctypes.byref(
                    _cfg(ins_threshold=2, pivot_policy=1, seed=r + 1)), st)),
                ("hoare", lambda a, st: L.orc_classical_sort(a.ctypes.data, n, I32, r + 1, st)),
                ("juggle", lambda a, st: L.orc_juggle_sort(a.ctypes.data, n, I32, r + 1, st)),
                ("full", lambda a, st: L.orc_tsqs_sort(a.ctypes.data, n, I32, ctypes.byref(
                    _cfg(seed=r + 1)), st))):
            if name == "full" and not full:
                continue
            a = x.copy()
            st = _Stats()
            call(a, ctypes.byref(st))
            if not (np.diff(a) == 1).all():
                raise AssertionError(f"{name} n={n}: not sorted")
            out[name] = (st.cmps, st.moves, st.swaps, st.stages)
        return out
    with ThreadPoolExecutor(threads) as ex:            # the oracle releases the GIL
        res = list(ex.map(one, range(reps)))
    keys = res[0].keys()
    return {k: dict(zip(("cmps", "moves", "swaps", "stages"),
                        np.mean([r[k] for r in res], axis=0))) for k in keys}


def whole_sort_fail(means: dict) -> str | None:
    """Checks means {n: whole_sort_means(n)} against eqs. (3), (4), (8), (9) and the 2/3
    relation; None if every pin holds."""
    ns = sorted(means)
    for n in ns:
        m = means[n]
        if abs(m["ts"]["cmps"] / eq3(n) - 1) > 0.05:
            return f"n={n}: Triple State comparisons / eq. (3) = {m['ts']['cmps'] / eq3(n):.4f}"
        if abs(m["hoare"]["cmps"] / eq3(n) - 1) > 0.03:
            return f"n={n}: Hoare comparisons / eq. (3) = {m['hoare']['cmps'] / eq3(n):.4f}"
        if abs(m["hoare"]["swaps"] / eq4(n) - 1) > 0.05:
            return f"n={n}: Hoare exchanges / eq. (4) = {m['hoare']['swaps'] / eq4(n):.4f}"
        if abs(m["juggle"]["moves"] / 3 / eq8(n) - 1) > 0.05:
            return f"n={n}: juggling virtual swaps / eq. (8) = {m['juggle']['moves'] / 3 / eq8(n):.4f}"
        r10 = (m["ts"]["moves"] - 5 * m["ts"]["stages"]) / (3 * eq8(n))
        if abs(r10 - 1) > (0.05 if n >= 10 ** 5 else 0.08):
            return f"n={n}: (Triple State copies - 5 per stage) / (3 eq. (8)) = {r10:.4f}"
    for a, b in zip(ns, ns[1:]):
        d = math.log(b) - math.log(a)

        def slope(k, f):
            return (means[b][k][f] / b - means[a][k][f] / a) / d
        checks = (("ts", "cmps", 1, 2.0, 0.05), ("hoare", "swaps", 1, 1 / 3, 0.03),
                  ("juggle", "moves", 3, 2 / 9, 0.05))
        for k, f, div, want, tol in checks:
            s = slope(k, f) / div
            if abs(s / want - 1) > tol:
                return f"{a}->{b}: n ln n coefficient of {k} {f} = {s:.4f}, expected {want:.4f}"
        ratio = slope("ts", "moves") / 3 / slope("hoare", "swaps")
        if not 0.60 <= ratio <= 0.80:
            return f"{a}->{b}: Triple State / Hoare n ln n ratio {ratio:.4f} outside [0.60, 0.80]"
    return None


@pytest.fixture(scope="module")
def whole_means(orc):
    L = bind(orc.lib())
    return {n: whole_sort_means(L, n, 200) for n in (10 ** 4, 10 ** 5, 10 ** 6)}


def test_whole_sort_counts_match_section_v_a(whole_means):
    assert whole_sort_fail(whole_means) is None


def test_two_thirds_relation_report(whole_means):
    """Reports the Triple State / classical ratios; the whole-sort ratio falls with n
    toward the ratio of the n ln n coefficients (the linear terms differ in sign)."""
    ns = sorted(whole_means)
    ratios = [whole_means[n]["ts"]["moves"] / 3 / whole_means[n]["hoare"]["swaps"] for n in ns]
    full = [whole_means[n]["full"]["moves"] / 3 / whole_means[n]["hoare"]["swaps"] for n in ns]
    print("random pivot, no insertion sort:", [round(r, 4) for r in ratios])
    print("full configuration:", [round(r, 4) for r in full])
    assert ratios[0] > ratios[1] > ratios[2]
    assert full[0] > full[1] > full[2]
    # the paper's configuration (sampled pivots, insertion sort) compares less than
    # the random-pivot quicksort of eq. (3)
    for n in ns:
        assert whole_means[n]["full"]["cmps"] < whole_means[n]["ts"]["cmps"]
