"""The N>1 path of bench.py runs independent replicas: no data-path collective, only
the barrier and the max/sum reductions of the timing.  Exercised here with two gloo
ranks on CPU (spawned processes, no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    d = bench.Dist(world)
    d.barrier()
    mx = d.max(float(rank + 1) * 10.0)          # slowest rank's time
    sm = d.sum(float(1000 * (rank + 1)))        # keys of all ranks
    d.barrier()
    d.close()
    out.put((rank, mx, sm))


def test_two_rank_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, mx, sm in res:
        assert mx == 20.0 and sm == 3000.0
