"""Planted mistakes: each is a plausible one-token slip in the oracle's C source.
The mutated copy is compiled on the CPU and must fail the brute-force pin, which
shows the pins are sharp enough to catch it.  Nothing here touches a GPU or the
committed oracle library."""
import ctypes
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from tests.test_oracle_pins import weak_orderings

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "tsqs_oracle.c")

MUTATIONS = {
    # State 3L evacuates an equal only while r is still inside the old run
    "3L_evacuation_bound": ("if (r >= ml) { ccopy(c, TAR(c, i), AR(c, r)); i++; }\n                } while",
                            "if (r > ml) { ccopy(c, TAR(c, i), AR(c, r)); i++; }\n                } while"),
    # exit of Section III.F: forgetting to exclude p from the left part
    "exit_no_l_decrement": ("ccopy(c, AR(c, l), P);\n                l--;",
                            "ccopy(c, AR(c, l), P);\n"),
    # State 2L roll: forgetting to move the last equal into m
    "2L_roll_missing": ("r--;\n                ccopy(c, AR(c, m), AR(c, r));\n                m--;\n                state = (m == l) ? S_EXIT2 : S_2L_M;",
                        "r--;\n                m--;\n                state = (m == l) ? S_EXIT2 : S_2L_M;"),
    # State 1: wrong direction when growing the run of equals
    "state1_gap_sign": ("if (r - mr > ml - l) { mr++; state = S_MR_SCAN1; }   /* larger gap */",
                        "if (r - mr < ml - l) { mr++; state = S_MR_SCAN1; }   /* larger gap */"),
    # copy-back of tar in State 3R moves the wrong way
    "3R_copyback_direction": ("while (i > 0) { i--; m--; ccopy(c, AR(c, m), TAR(c, i)); }",
                              "while (i > 0) { i--; m++; ccopy(c, AR(c, m), TAR(c, i)); }"),
    # late swapping (VIII.H): equal keys no longer ordered by their original place
    "wide_tie_unstable": ("return px < py ? -1 : (px > py ? 1 : 0);", "return 0;"),
    # late swapping: a cycle member not marked placed is walked again
    "wide_cycle_unmarked": ("            placed[src] = 1;\n", ""),
    # counters: the insertion sort (Section IV) counts its copy into temp twice
    "insertion_double_count": ("ccopy(c, c->temp, AR(c, j));",
                               "ccopy(c, c->temp, AR(c, j)); c->st->moves++;"),
    # counters: the median-of-five insertion over the sample positions counts a copy twice
    "pivot_double_count": ("ccopy(c, c->scratch, AR(c, pos[s]));",
                           "ccopy(c, c->scratch, AR(c, pos[s])); c->st->moves++;"),
    # counters: State 1 counts the copy of a larger element into the hole at r twice
    "stage_double_count": ("ccopy(c, AR(c, r), AR(c, l));\n                r--;\n                state = (mr == r)",
                           "ccopy(c, AR(c, r), AR(c, l)); c->st->moves++;\n                r--;\n                state = (mr == r)"),
}


def _build_mutant(name, tmpdir):
    old, new = MUTATIONS[name] if name else ("", "")
    src = open(SRC).read()
    assert not name or src.count(old) == 1, f"mutation site for {name} not unique"
    path = os.path.join(tmpdir, f"m_{name}.c")
    open(path, "w").write(src.replace(old, new) if name else src)
    hdr_dir = os.path.dirname(SRC)
    so = os.path.join(tmpdir, f"m_{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-I", hdr_dir,
                           "-o", so, path, "-lpthread"])
    return ctypes.CDLL(so)


def _exhaustive_fails(L) -> bool:
    from oracle.oracle import _Cfg, _Stats
    L.orc_tsqs_sort_rows.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                     ctypes.c_int, ctypes.POINTER(_Cfg), ctypes.POINTER(_Stats)]
    for n in range(3, 8):
        w = weak_orderings(n)
        for policy in (0, 1):
            a = np.ascontiguousarray(w.copy())
            cfg = _Cfg(2, policy, 1, 70, 800, 40000, 1)
            st = _Stats()
            L.orc_tsqs_sort_rows(a.ctypes.data, len(w), n, 1, ctypes.byref(cfg), ctypes.byref(st))
            if not np.array_equal(a, np.sort(w, axis=1)):
                return True
    # larger arrays with few distinct values reach State 3L/3R with a non-empty run
    rng = np.random.default_rng(11)
    for n in (8, 9, 12, 20, 40, 100, 300):
        for k in (2, 3, 5, 9, 30):
            rows = rng.integers(0, k, (200, n)).astype(np.int32)
            for policy in (0, 1):
                a = np.ascontiguousarray(rows.copy())
                cfg = _Cfg(2, policy, 1, 70, 800, 40000, 1)
                st = _Stats()
                L.orc_tsqs_sort_rows(a.ctypes.data, len(rows), n, 1, ctypes.byref(cfg), ctypes.byref(st))
                if not np.array_equal(a, np.sort(rows, axis=1)):
                    return True
    # one stage must leave exactly <p | =p | >p and exclude the whole =p run (III.F)
    L.orc_tsqs_stage.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_size_t,
                                 ctypes.POINTER(_Stats), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_longlong)]
    for n in (3, 5, 9, 33, 257):
        for _ in range(50):
            x = rng.integers(0, 4, n).astype(np.int32)
            pi = int(rng.integers(0, n))
            p = x[pi]
            a = x.copy()
            st, lo, hi = _Stats(), ctypes.c_longlong(), ctypes.c_longlong()
            L.orc_tsqs_stage(a.ctypes.data, n, 1, pi, ctypes.byref(st), ctypes.byref(lo), ctypes.byref(hi))
            lo, hi = lo.value, hi.value
            if not ((a[:lo + 1] < p).all() and (a[hi:] > p).all() and (a[lo + 1:hi] == p).all()):
                return True
    # late swapping of wide elements against the stable order (few distinct keys)
    from tests.test_oracle_wide import _expected, _make
    L.orc_wide_sort.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_size_t,
                                ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                ctypes.POINTER(ctypes.c_uint64)]
    for n, es, off in ((7, 12, 0), (100, 16, 4), (1000, 24, 8)):
        raw = _make(n, es, off, 1, seed=n, distinct=5)
        got = raw.copy()
        mv, cy = ctypes.c_uint64(), ctypes.c_uint64()
        L.orc_wide_sort(got.ctypes.data, n, es, off, 1, ctypes.byref(mv), ctypes.byref(cy))
        if got.tobytes() != _expected(raw, n, es, off, np.int32).tobytes():
            return True
    return False


def _counts_fail(L) -> bool:
    """The counter pins of tests/test_oracle_counts.py, the whole-sort ones at reduced
    size (40 permutations at n = 10^4 and 10^5)."""
    from tests.test_oracle_counts import (bind, insertion_sort_counts_fail, pivot_counts_fail,
                                          whole_sort_fail, whole_sort_means)
    bind(L)
    if insertion_sort_counts_fail(L) or pivot_counts_fail(L):
        return True
    means = {n: whole_sort_means(L, n, 40, full=False) for n in (10 ** 4, 10 ** 5)}
    return whole_sort_fail(means) is not None


def _run_child(name: str) -> int:
    """Child process: exit 0 if the mutant passes every check (escaped), 1 if a check
    failed.  A mutant that crashes or loops ends the child some other way."""
    with tempfile.TemporaryDirectory() as d:
        L = _build_mutant(name, d)
        return 1 if (_exhaustive_fails(L) or _counts_fail(L)) else 0


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    root = os.path.dirname(os.path.dirname(SRC))
    code = ("import sys; sys.path.insert(0, %r); from tests.test_oracle_mutations import _run_child; "
            "sys.exit(_run_child(%r))" % (root, name))
    try:
        rc = subprocess.run([sys.executable, "-c", code], timeout=120,
                            capture_output=True).returncode
    except subprocess.TimeoutExpired:
        rc = -1                                   # the mutant looped: caught
    assert rc != 0, f"mutation {name} escaped the pins"


def test_unmutated_oracle_passes_every_check():
    """Control: the same checks on an unmutated copy all pass, so a caught mutant is
    caught by its mistake and not by a check that fails anyway."""
    root = os.path.dirname(os.path.dirname(SRC))
    code = ("import sys; sys.path.insert(0, %r); from tests.test_oracle_mutations import _run_child; "
            "sys.exit(_run_child(''))" % root)
    rc = subprocess.run([sys.executable, "-c", code], timeout=300, capture_output=True).returncode
    assert rc == 0
