"""Large elements on the GPU (tsqs_sort_wide) against the oracle's late swapping
(Section VIII.H): the result is the stable order by key, compared byte for byte."""
import ctypes

import numpy as np
import pytest

from tests.test_oracle_wide import KEY_TYPES, _make

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


SHAPES = [(8, 0), (12, 4), (16, 8), (24, 8), (56, 16), (320, 256)]


@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("es,off", SHAPES)
@pytest.mark.parametrize("n", [2, 4097, 100_003])
def test_wide_matches_oracle(T, orc, kind, es, off, n):
    ks = np.dtype(KEY_TYPES[kind]).itemsize
    if off + ks > es - 4 or off % ks or es % ks:
        pytest.skip("key does not fit before the index word")
    for distinct in (2**40, 9):
        raw = _make(n, es, off, kind, seed=n + es + kind, distinct=distinct)
        exp = raw.copy()
        orc.wide_sort(exp, es, off, kind)
        t = torch.from_numpy(raw.copy()).cuda()
        T.sort_wide_(t, es, off, kind)
        torch.cuda.synchronize()
        assert T.last_device_status() == 0
        assert t.cpu().numpy().tobytes() == exp.tobytes()


def test_wide_large_case(T, orc):
    n, es, off, kind = 1 << 21, 56, 8, 6
    raw = _make(n, es, off, kind, seed=3)
    exp = raw.copy()
    orc.wide_sort(exp, es, off, kind)
    t = torch.from_numpy(raw.copy()).cuda()
    T.sort_wide_(t, es, off, kind)
    torch.cuda.synchronize()
    assert T.last_device_status() == 0
    assert t.cpu().numpy().tobytes() == exp.tobytes()


def test_wide_argument_errors(T):
    t = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    L = T.lib()
    assert L.tsqs_sort_wide(p, 100, 10, 0, 1, None) == T.TSQS_EINVAL      # size not a multiple of 4
    assert L.tsqs_sort_wide(p, 100, 12, 4, 4, None) == T.TSQS_EINVAL      # 8-byte key in 12 bytes
    assert L.tsqs_sort_wide(p, 100, 16, 12, 4, None) == T.TSQS_EINVAL     # key past the element end
    assert L.tsqs_sort_wide(p, 100, 16, 0, 7, None) == T.TSQS_EINVAL      # records are not a key kind
    assert L.tsqs_sort_wide(ctypes.c_void_p(t.data_ptr() + 2), 100, 16, 0, 1, None) == T.TSQS_EINVAL
    assert L.tsqs_sort_wide(p, 1, 16, 0, 1, None) == T.TSQS_OK            # nothing to do
