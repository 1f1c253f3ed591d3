"""tsqs_sort_noalloc: the sort entry point for callers that cannot allocate device
memory when they sort (their device memory belongs to another allocator, or every
byte is budgeted up front, or a possibly synchronising cudaMalloc is too slow for
them).  Its output must equal the CPU oracle's and tsqs_sort's byte for byte (the
sorted output is unique), on consecutive calls that share its static scratch; a call
after the first must not change the device's free memory; it must refuse arrays above
its stated limit and a stream that is being captured.  This file is collected last,
and each test also passes when run alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle as orc
from workloads import int32_pattern, records_u64, floats_normal_specials

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MAX_BYTES = 16 << 20          # TSQS_NOALLOC_MAX_BYTES


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


def _expected(host: np.ndarray, kind: int) -> bytes:
    exp = host.copy()
    orc.tsqs_sort(exp, kind)
    return exp.tobytes()


def _noalloc(T, host: np.ndarray, kind: int, es: int) -> bytes:
    t = torch.from_numpy(host.view(np.int64) if es == 16 else host.copy()).cuda()
    s = torch.cuda.current_stream()
    rc = T.lib().tsqs_sort_noalloc(ctypes.c_void_p(t.data_ptr()), host.nbytes // es, es, kind,
                                   ctypes.c_void_p(s.cuda_stream))
    torch.cuda.synchronize()
    assert rc == T.TSQS_OK
    return t.cpu().numpy().tobytes()


def _tsqs_sort(T, host: np.ndarray, kind: int, es: int) -> bytes:
    t = torch.from_numpy(host.view(np.int64) if es == 16 else host.copy()).cuda()
    s = torch.cuda.current_stream()
    assert T.lib().tsqs_sort(ctypes.c_void_p(t.data_ptr()), host.nbytes // es, es, kind,
                             ctypes.c_void_p(s.cuda_stream)) == T.TSQS_OK
    torch.cuda.synchronize()
    assert T.last_device_status() == T.TSQS_OK
    return t.cpu().numpy().tobytes()


CASES = [
    ("int32 random", lambda: int32_pattern("random", 1_000_003, seed=1), 1, 4),
    ("int32 many equals", lambda: int32_pattern("many_equals", 3_000_001, seed=2), 1, 4),
    ("float32 specials", lambda: floats_normal_specials(700_001, seed=3, special_frac=0.01), 3, 4),
    ("float32 small", lambda: floats_normal_specials(65_537, seed=4, special_frac=0.05), 3, 4),
    ("records", lambda: records_u64(300_001, seed=5), 7, 16),
    ("records at the limit", lambda: records_u64(1 << 20, seed=6), 7, 16),
]


def test_noalloc_equals_oracle_and_tsqs_sort_on_consecutive_calls(T):
    # two calls in a row per case: the second sees whatever the first left behind
    for name, make, kind, es in CASES:
        host = make()
        exp = _expected(host, kind)
        assert _tsqs_sort(T, host, kind, es) == exp, name
        for _ in range(2):
            assert _noalloc(T, host, kind, es) == exp, name


def test_noalloc_largest_int32_twice_allocates_nothing(T):
    n = MAX_BYTES // 4
    host = [int32_pattern("random", n, seed=seed) for seed in (7, 8)]
    t = [torch.from_numpy(h.copy()).cuda() for h in host]
    s = torch.cuda.current_stream()
    L = T.lib()
    # the first call on the device does the set-up
    assert L.tsqs_sort_noalloc(ctypes.c_void_p(t[0].data_ptr()), n, 4, 1,
                               ctypes.c_void_p(s.cuda_stream)) == T.TSQS_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert L.tsqs_sort_noalloc(ctypes.c_void_p(t[1].data_ptr()), n, 4, 1,
                               ctypes.c_void_p(s.cuda_stream)) == T.TSQS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for h, d in zip(host, t):
        assert d.cpu().numpy().tobytes() == _expected(h, orc.KIND_I32)


def test_noalloc_rejects_arrays_over_the_limit(T):
    n = MAX_BYTES // 4 + 1
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    rc = T.lib().tsqs_sort_noalloc(ctypes.c_void_p(t.data_ptr()), n, 4, 1, ctypes.c_void_p(s.cuda_stream))
    assert rc == T.TSQS_EINVAL
    assert int(t.abs().sum().item()) == 0          # nothing was touched


def test_noalloc_refuses_a_capturing_stream(T):
    host = int32_pattern("random", 4097, seed=9)
    t = torch.from_numpy(host.copy()).cuda()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    dummy = torch.zeros(1, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g.capture_begin()
        dummy.add_(1)                                     # the capture is not empty
        rc = T.lib().tsqs_sort_noalloc(ctypes.c_void_p(t.data_ptr()), len(host), 4, 1,
                                       ctypes.c_void_p(s.cuda_stream))
        g.capture_end()
    assert rc == T.TSQS_EINVAL
    torch.cuda.synchronize()
    assert t.cpu().numpy().tobytes() == host.tobytes()     # nothing was queued
    # the device and the entry point are still usable
    assert _noalloc(T, host, 1, 4) == _expected(host, orc.KIND_I32)
