"""tsqs_sort_noalloc: the sort entry point for callers that cannot allocate device
memory when they sort (their memory belongs to another allocator, or every byte is
budgeted up front, or a possibly synchronising cudaMalloc is too slow for them).  It
must give exactly what tsqs_sort gives -- the sorted output is unique, so the
comparison is byte for byte -- on consecutive calls that share its static scratch,
and it must refuse arrays above its stated limit.  This file is collected last."""
import ctypes

import numpy as np
import pytest

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


def _both(T, host: np.ndarray, kind: int, es: int):
    """Sorts the same input with tsqs_sort and with tsqs_sort_noalloc."""
    src = torch.from_numpy(host.view(np.int64) if es == 16 else host.copy()).cuda()
    a = src.clone()
    b = src.clone()
    s = torch.cuda.current_stream()
    L = T.lib()
    n = host.nbytes // es
    assert L.tsqs_sort(ctypes.c_void_p(a.data_ptr()), n, es, kind, ctypes.c_void_p(s.cuda_stream)) == 0
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    rc = L.tsqs_sort_noalloc(ctypes.c_void_p(b.data_ptr()), n, es, kind, ctypes.c_void_p(s.cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0
    return a.cpu().numpy().tobytes(), b.cpu().numpy().tobytes()


def test_noalloc_equals_tsqs_sort_on_consecutive_calls(T):
    # two calls in a row per kind: the second sees whatever the first left behind
    cases = [
        (int32_pattern("random", 1_000_003, seed=1), 1, 4),
        (int32_pattern("many_equals", 3_000_001, seed=2), 1, 4),
        (floats_normal_specials(700_001, seed=3, special_frac=0.01), 3, 4),
        (floats_normal_specials(65_537, seed=4, special_frac=0.05), 3, 4),
        (records_u64(300_001, seed=5), 7, 16),
        (records_u64(1 << 20, seed=6), 7, 16),              # exactly the limit
    ]
    for host, kind, es in cases:
        ref, got = _both(T, host, kind, es)
        assert ref == got


def test_noalloc_largest_int32_twice(T):
    n = MAX_BYTES // 4
    for seed in (7, 8):
        ref, got = _both(T, int32_pattern("random", n, seed=seed), 1, 4)
        assert ref == got


def test_noalloc_rejects_arrays_over_the_limit(T):
    n = MAX_BYTES // 4 + 1
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    rc = T.lib().tsqs_sort_noalloc(ctypes.c_void_p(t.data_ptr()), n, 4, 1, ctypes.c_void_p(s.cuda_stream))
    assert rc == T.TSQS_EINVAL
    assert int(t.abs().sum().item()) == 0          # nothing was touched
