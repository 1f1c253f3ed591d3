"""Host arrays streamed through the GPU (tsqs_ctx_sort_host_stream): every item, sorted
in place or into its own output array, equals the oracle's sort (Section III, the
qsort() of an array in host memory); staging slots are reused past three items and
regrown for larger items; page-locked and pageable host memory; argument errors queue
nothing."""
import ctypes

import numpy as np
import pytest

from workloads import int32_pattern, records_u64, floats_normal_specials

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


def _oracle(orc, a, kind):
    b = np.ascontiguousarray(a.copy())
    orc.tsqs_sort(b, kind)
    return b


SIZES = [0, 1, 2, 4097, 100_003, 3, 1_000_001, 65_536, 17, 300_000]
PATTERNS = ["random", "random", "sorted", "random", "reversed", "random", "many_equals",
            "organ_pipe", "random", "stair_steps"]


@pytest.mark.parametrize("pinned", [True, False])
def test_stream_int32_out_of_place(T, orc, pinned):
    arrs = [int32_pattern(p, n, seed=i + 1) for i, (p, n) in enumerate(zip(PATTERNS, SIZES))]
    ins = [torch.from_numpy(a.copy()) for a in arrs]
    outs = [torch.empty_like(t) for t in ins]
    if pinned:
        ins = [t.pin_memory() for t in ins]
        outs = [t.pin_memory() for t in outs]
    ctx = T.Context()
    st = ctx.sort_host_stream(ins, outs, kind=T.TSQS_I32)
    assert st == [0] * len(SIZES)
    for a, t_in, t_out in zip(arrs, ins, outs):
        assert t_in.numpy().tobytes() == a.tobytes()            # inputs left as they were
        assert t_out.numpy().tobytes() == _oracle(orc, a, 1).tobytes()
    ctx.close()


def test_stream_in_place_kinds_and_regrowth(T, orc):
    ctx = T.Context()
    # small items first, then larger ones: the staging slots grow between calls
    for scale in (1, 7):
        f = [floats_normal_specials(n * scale, seed=n + scale) for n in (5, 40_000, 9_001, 70_000)]
        tf = [torch.from_numpy(a.copy()).pin_memory() for a in f]
        assert ctx.sort_host_stream(tf, kind=T.TSQS_F32) == [0] * len(f)
        for a, t in zip(f, tf):
            assert t.numpy().view(np.float32).tobytes() == _oracle(orc, a, 3).tobytes()
        r = [records_u64(n * scale, seed=n) for n in (3, 20_001, 4096, 50_000, 2)]
        tr = [torch.from_numpy(a.view(np.int64).copy()) for a in r]
        assert ctx.sort_host_stream(tr, kind=T.TSQS_U64_U64_REC) == [0] * len(r)
        for a, t in zip(r, tr):
            assert t.numpy().view(np.uint64).reshape(-1, 2).tobytes() == _oracle(orc, a, 7).tobytes()
        x = [((np.arange(n, dtype=np.int64) * 7919) % 100_003 - 50_000) * (1 << 33)
             for n in (60_000 * scale, 1, 4100)]
        tx = [torch.from_numpy(a.copy()).pin_memory() for a in x]
        assert ctx.sort_host_stream(tx, kind=T.TSQS_I64) == [0] * len(x)
        for a, t in zip(x, tx):
            assert t.numpy().tobytes() == _oracle(orc, a, 4).tobytes()
    ctx.close()


def test_stream_many_items_one_input(T, orc):
    """The same host input streamed into several outputs (the end-to-end bench's use)."""
    a = int32_pattern("random", 2_000_003, seed=11)
    src = torch.from_numpy(a.copy()).pin_memory()
    outs = [torch.empty_like(src).pin_memory() for _ in range(3)]
    ctx = T.Context()
    st = ctx.sort_host_stream([src] * 8, [outs[i % 3] for i in range(8)], kind=T.TSQS_I32)
    assert st == [0] * 8
    exp = _oracle(orc, a, 1).tobytes()
    for o in outs:
        assert o.numpy().tobytes() == exp
    assert src.numpy().tobytes() == a.tobytes()
    ctx.close()


def test_stream_argument_errors(T):
    L = T.lib()
    ctx = T.Context()
    buf = torch.zeros(64, dtype=torch.int32)
    p = (ctypes.c_void_p * 2)(buf.data_ptr(), buf.data_ptr())
    sizes = (ctypes.c_size_t * 2)(64, 64)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.tsqs_ctx_sort_host_stream(ctx.handle, p, None, sizes, 2, 8, T.TSQS_I32, s, None) == T.TSQS_EINVAL
    assert L.tsqs_ctx_sort_host_stream(ctx.handle, p, None, sizes, 2, 4, 99, s, None) == T.TSQS_EINVAL
    big = (ctypes.c_size_t * 2)(64, 1 << 31)
    assert L.tsqs_ctx_sort_host_stream(ctx.handle, p, None, big, 2, 4, T.TSQS_I32, s, None) == T.TSQS_EINVAL
    nul = (ctypes.c_void_p * 2)(buf.data_ptr(), None)
    assert L.tsqs_ctx_sort_host_stream(ctx.handle, nul, None, sizes, 2, 4, T.TSQS_I32, s, None) == T.TSQS_EINVAL
    assert L.tsqs_ctx_sort_host_stream(ctx.handle, None, None, None, 0, 4, T.TSQS_I32, s, None) == T.TSQS_OK
    assert L.tsqs_ctx_sort_host_stream(None, p, None, sizes, 2, 4, T.TSQS_I32, s, None) == T.TSQS_EINVAL
    ctx.close()
