"""tsqs_graph_sort_segmented: the caller-held graph of a whole sort (capture once,
replay).  The first call builds and launches the graph; later calls with the same
handle update its setup node for new arrays and relaunch it; the caller may replay it
directly with cudaGraphLaunch.  Every result is compared with the oracle byte for byte
(marked gpu)."""
import ctypes
import os

import numpy as np
import pytest

from workloads import int32_pattern, floats_normal_specials
from workloads.patterns import batched_segments, batched_keys

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


def _cudart():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    L = ctypes.CDLL(os.path.join(home, "lib64", "libcudart.so"))
    L.cudaGraphLaunch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.cudaGraphLaunch.restype = ctypes.c_int
    return L


def _oracle_segments(orc, x, offs):
    exp = x.copy()
    orc.tsqs_sort_segments(exp, offs, orc.KIND_I32, threads=8)
    return exp.tobytes()


def test_graph_build_update_and_replay_segmented(T, orc):
    offs, sizes, pat = batched_segments(1500, seed=21, max_log2=15)
    d_offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    total = int(offs[-1])
    ctx = T.Context()
    ctx.reserve(total, len(sizes), 4)
    # first call: build, instantiate, launch
    x1 = batched_keys(offs, pat, seed=21)
    t = torch.from_numpy(x1.copy()).cuda()
    h = ctx.graph_sort_segmented(t, d_offs, kind=T.TSQS_I32)
    assert h
    assert ctx.status() == T.TSQS_OK
    assert t.cpu().numpy().tobytes() == _oracle_segments(orc, x1, offs)
    # second call, new contents in a new buffer: the same graph, its setup node updated
    x2 = batched_keys(offs, pat, seed=22)
    t2 = torch.from_numpy(x2.copy()).cuda()
    h2 = ctx.graph_sort_segmented(t2, d_offs, h, kind=T.TSQS_I32)
    assert h2 == h
    assert ctx.status() == T.TSQS_OK
    assert t2.cpu().numpy().tobytes() == _oracle_segments(orc, x2, offs)
    # direct replay by the caller: refill t2 and launch the graph as it stands
    x3 = batched_keys(offs, pat, seed=23)
    t2.copy_(torch.from_numpy(x3))
    s = torch.cuda.current_stream()
    assert _cudart().cudaGraphLaunch(ctypes.c_void_p(h), ctypes.c_void_p(s.cuda_stream)) == 0
    torch.cuda.synchronize()
    assert ctx.status() == T.TSQS_OK
    assert t2.cpu().numpy().tobytes() == _oracle_segments(orc, x3, offs)
    # other segment boundaries (fewer segments) through the same handle
    offs_b = offs[::3].copy()
    offs_b[-1] = offs[-1]
    d_offs_b = torch.from_numpy(offs_b.astype(np.int64)).cuda()
    t3 = torch.from_numpy(x1.copy()).cuda()
    assert ctx.graph_sort_segmented(t3, d_offs_b, h, kind=T.TSQS_I32) == h
    assert ctx.status() == T.TSQS_OK
    assert t3.cpu().numpy().tobytes() == _oracle_segments(orc, x1, offs_b)
    # a handle made for int32 is refused for another key kind
    f = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(T.TsqsError):
        ctx.graph_sort_segmented(f, None, h, kind=T.TSQS_F32)
    ctx.graph_destroy(h)
    ctx.close()


def test_graph_single_segment_kinds(T, orc):
    ctx = T.Context()
    a = int32_pattern("random", (1 << 20) + 3, seed=24)
    t = torch.from_numpy(a.copy()).cuda()
    h = ctx.graph_sort_segmented(t, None, kind=T.TSQS_I32)
    assert ctx.status() == T.TSQS_OK
    exp = a.copy()
    orc.tsqs_sort(exp, orc.KIND_I32)
    assert t.cpu().numpy().tobytes() == exp.tobytes()
    b = floats_normal_specials(300_001, seed=25, special_frac=0.01)
    tb = torch.from_numpy(b.copy()).cuda()
    hf = ctx.graph_sort_segmented(tb, None, kind=T.TSQS_F32)
    assert hf and hf != h
    assert ctx.status() == T.TSQS_OK
    expb = b.copy()
    orc.tsqs_sort(expb, orc.KIND_F32)
    assert tb.cpu().numpy().tobytes() == expb.tobytes()
    # a smaller array through the int32 handle
    c = int32_pattern("many_equals", 70_001, seed=26)
    tc = torch.from_numpy(c.copy()).cuda()
    assert ctx.graph_sort_segmented(tc, None, h, kind=T.TSQS_I32) == h
    assert ctx.status() == T.TSQS_OK
    expc = c.copy()
    orc.tsqs_sort(expc, orc.KIND_I32)
    assert tc.cpu().numpy().tobytes() == expc.tobytes()
    ctx.close()                                   # releases both graphs


def test_graph_follows_the_schedule_bound(T, orc):
    """A held graph is built for the schedule its size takes (task-parallel up to 2^24
    elements by default): a later call across the bound releases it and returns the
    other graph's handle; direct replays of either give the oracle's result."""
    ctx = T.Context()
    small = int32_pattern("random", 200_003, seed=31)
    t = torch.from_numpy(small.copy()).cuda()
    h1 = ctx.graph_sort_segmented(t, None, kind=T.TSQS_I32)
    assert h1 and ctx.status() == T.TSQS_OK
    exp_small = small.copy()
    orc.tsqs_sort(exp_small, orc.KIND_I32)
    assert t.cpu().numpy().tobytes() == exp_small.tobytes()
    t.copy_(torch.from_numpy(small))
    s = torch.cuda.current_stream()
    assert _cudart().cudaGraphLaunch(ctypes.c_void_p(h1), ctypes.c_void_p(s.cuda_stream)) == 0
    torch.cuda.synchronize()
    assert ctx.status() == T.TSQS_OK
    assert t.cpu().numpy().tobytes() == exp_small.tobytes()
    # past the bound: the level-by-level graph under a new handle
    big = torch.from_numpy(int32_pattern("random", (1 << 24) + 4099, seed=32)).cuda()
    ref = torch.sort(big)[0]
    h2 = ctx.graph_sort_segmented(big, None, h1, kind=T.TSQS_I32)
    assert h2 and ctx.status() == T.TSQS_OK
    assert torch.equal(big, ref)
    # and back below it
    t2 = torch.from_numpy(small.copy()).cuda()
    h3 = ctx.graph_sort_segmented(t2, None, h2, kind=T.TSQS_I32)
    assert h3 and ctx.status() == T.TSQS_OK
    assert t2.cpu().numpy().tobytes() == exp_small.tobytes()
    ctx.graph_destroy(h3)
    ctx.close()
