"""Batching (segmented sort under one graph, autotuned plans) and serving
(continuous batching of requests) against the oracle (marked gpu)."""
import ctypes

import numpy as np
import pytest

from workloads import PATTERNS, int32_pattern, records_u64
from workloads.patterns import batched_segments, batched_keys, serving_requests

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


def test_autotune_returns_working_plan(T, orc):
    plan = T.Plan()
    s = torch.cuda.current_stream()
    rc = T.lib().tsqs_plan_autotune(1, 1 << 21, 1, ctypes.c_void_p(s.cuda_stream), ctypes.byref(plan))
    assert rc == 0
    assert plan.small_threshold in (1024, 2048, 4096) and plan.sample_count in (15, 31, 63)
    again = T.Plan()
    assert T.lib().tsqs_plan_default(1, 1 << 21, ctypes.byref(again)) == 0
    assert (again.small_threshold, again.sample_count, again.tile_items) == \
        (plan.small_threshold, plan.sample_count, plan.tile_items)
    ctx = T.Context(plan)
    a = int32_pattern("random", 1 << 21, seed=9)
    t = torch.from_numpy(a.copy()).cuda()
    T.sort_(t, kind=1, ctx=ctx)
    assert ctx.status() == 0
    exp = a.copy()
    orc.tsqs_sort(exp, 1)
    assert t.cpu().numpy().tobytes() == exp.tobytes()


def test_batched_graph_replay_twice_identical(T, orc):
    """The segmented sort replays the same captured graph on every call; two replays
    on the same input give identical bytes, equal to per-segment oracle sorts."""
    offs, sizes, pat = batched_segments(2000, seed=4, max_log2=14)
    x = batched_keys(offs, pat, seed=4)
    d_offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    ctx = T.Context()
    outs = []
    for _ in range(2):
        t = torch.from_numpy(x.copy()).cuda()
        T.sort_segmented_(t, d_offs, kind=1, ctx=ctx)
        assert ctx.status() == 0
        outs.append(t.cpu().numpy())
    exp = x.copy()
    orc.tsqs_sort_segments(exp, offs, 1, threads=4)
    assert outs[0].tobytes() == outs[1].tobytes() == exp.tobytes()


def test_batched_equals_per_call(T):
    """Every segment sorted in the batch equals the same segment sorted alone."""
    offs, sizes, pat = batched_segments(300, seed=6, max_log2=16)
    x = batched_keys(offs, pat, seed=6)
    t = torch.from_numpy(x.copy()).cuda()
    T.sort_segmented_(t, torch.from_numpy(offs.astype(np.int64)).cuda(), kind=1)
    alone = torch.from_numpy(x.copy()).cuda()
    for s in range(300):
        lo, hi = int(offs[s]), int(offs[s + 1])
        if hi > lo:
            T.sort_(alone[lo:hi], kind=1)
    torch.cuda.synchronize()
    assert torch.equal(t, alone)


def test_server_mixed_requests_match_alone(T, orc):
    L = T.lib()
    srv = L.tsqs_server_create(1 << 30, 3, 64)
    assert srv
    req = serving_requests(120, seed=3, lo_log2=6, hi_log2=21)
    bufs, inputs, kinds, tickets = [], [], [], []
    try:
        for i in range(120):
            n = int(req["sizes"][i])
            pat = PATTERNS[int(req["pattern"][i])]
            if req["is_rec"][i]:
                a = records_u64(n, seed=i)
                t = torch.from_numpy(a.view(np.int64).copy()).cuda()
                kind, es = 7, 16
            else:
                a = int32_pattern(pat, n, seed=i)
                t = torch.from_numpy(a.copy()).cuda()
                kind, es = 1, 4
            bufs.append(t); inputs.append(a); kinds.append(kind)
        torch.cuda.synchronize()
        # arrivals in bursts of 20: lanes are busy when the next burst lands, so later
        # requests queue and are packed into batches
        for i, (t, a, kind) in enumerate(zip(bufs, inputs, kinds)):
            tk = ctypes.c_uint64()
            es = 16 if kind == 7 else 4
            assert L.tsqs_server_submit(srv, ctypes.c_void_p(t.data_ptr()), len(a), es, kind,
                                        ctypes.byref(tk)) == 0
            tickets.append(tk.value)
            if i % 20 == 19:
                L.tsqs_server_progress(srv)
        assert L.tsqs_server_drain(srv) == 0
        batched = 0
        for t, a, kind, tk in zip(bufs, inputs, kinds, tickets):
            res = T.Result()
            assert L.tsqs_server_poll(srv, tk, ctypes.byref(res)) == 0
            assert res.done == 1 and res.status == 0
            assert res.t_submit <= res.t_start <= res.t_done
            batched += res.batch_size > 1
            exp = np.ascontiguousarray(a.copy())
            orc.tsqs_sort(exp, kind)
            got = t.cpu().numpy()
            assert got.tobytes() == exp.tobytes()
        assert batched > 0, "no request was batched with another"
    finally:
        L.tsqs_server_destroy(srv)


def test_server_rejects_oversize_and_bad_args(T):
    L = T.lib()
    srv = L.tsqs_server_create(64 << 20, 2, 8)
    assert srv
    try:
        t = torch.zeros(1 << 24, dtype=torch.int32, device="cuda")
        tk = ctypes.c_uint64()
        assert L.tsqs_server_submit(srv, ctypes.c_void_p(t.data_ptr()), 1 << 24, 4, 1,
                                    ctypes.byref(tk)) == T.TSQS_ENOMEM
        assert L.tsqs_server_submit(srv, ctypes.c_void_p(t.data_ptr()), 16, 8, 1,
                                    ctypes.byref(tk)) == T.TSQS_EINVAL
    finally:
        L.tsqs_server_destroy(srv)
