"""The records leaf sorts 64-bit packed keys ((key - min) >> sh << 12 | index) and puts
runs of equal packed keys in (key, payload) order from the records, with an indirect
network for runs longer than 32.  Inputs that drive every branch -- key ranges wider
than 2^52 (sh > 0: keys that differ only in dropped bits tie), long runs of equal keys,
equal keys with distinct payloads, exact duplicates -- are compared with the oracle
byte for byte, through the leaf kernel alone (every segment <= 4096 records) and
through the whole sort (marked gpu)."""
import ctypes

import numpy as np
import pytest

from workloads import rand_u64

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


def _records(kind: str, n: int, seed: int) -> np.ndarray:
    key = rand_u64(seed, 70, n)
    pay = rand_u64(seed, 71, n)
    r = np.empty((n, 2), dtype=np.uint64)
    if kind == "wide":             # full 64-bit range: sh = 12
        r[:, 0] = key
    elif kind == "wide_low_ties":  # keys equal above bit 12, distinct below: ties after the shift
        r[:, 0] = (key & np.uint64(0xF000000000000000)) | (key & np.uint64(0xFFF))
    elif kind == "all_equal":      # one run of the whole item: the indirect network
        r[:, 0] = np.uint64(0x0123456789ABCDEF)
    elif kind == "few_keys":       # runs of ~n/5 equal keys with distinct payloads
        r[:, 0] = key % np.uint64(5)
    elif kind == "runs_33":        # runs of exactly 33 equal keys (just past the short-run fix-up)
        r[:, 0] = (np.arange(n, dtype=np.uint64) // np.uint64(33)) * np.uint64(1 << 40)
        r = r[np.random.default_rng(seed).permutation(n)]
        r[:, 1] = pay
        return np.ascontiguousarray(r)
    elif kind == "dups":           # exact duplicate records among near keys
        r[:, 0] = key >> np.uint64(50)
        pay = pay % np.uint64(3)
    else:
        raise ValueError(kind)
    r[:, 1] = pay
    return r


KINDS = ["wide", "wide_low_ties", "all_equal", "few_keys", "runs_33", "dups"]


def _expected(orc, r: np.ndarray, offs=None) -> bytes:
    exp = r.copy()
    if offs is None:
        orc.tsqs_sort(exp, orc.KIND_REC)
    else:
        orc.tsqs_sort_segments(exp, offs, orc.KIND_REC, threads=8)
    return exp.tobytes()


@pytest.mark.parametrize("kind", KINDS)
def test_records_leaf_alone(T, orc, kind):
    sizes = [1, 2, 31, 32, 33, 100, 511, 512, 1000, 2049, 3000, 4095, 4096]
    offs = np.zeros(len(sizes) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(sizes)
    n = int(offs[-1])
    r = _records(kind, n, seed=len(kind))
    t = torch.from_numpy(r.view(np.int64).copy()).cuda()
    d_offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    s = torch.cuda.current_stream()
    assert T.lib().tsqs_debug_small_sort(ctypes.c_void_p(t.data_ptr()), n, 16, T.TSQS_U64_U64_REC,
                                         ctypes.c_void_p(d_offs.data_ptr()), len(sizes),
                                         ctypes.c_void_p(s.cuda_stream)) == 0
    assert T.last_device_status() == 0
    assert t.cpu().numpy().tobytes() == _expected(orc, r, offs)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [4097, 300_001])
def test_records_whole_sort(T, orc, kind, n):
    r = _records(kind, n, seed=n % 97)
    t = torch.from_numpy(r.view(np.int64).copy()).cuda()
    T.sort_(t, kind=T.TSQS_U64_U64_REC)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    assert t.cpu().numpy().tobytes() == _expected(orc, r)
