"""Multi-rank host logic of bench.py on CPU: two gloo ranks (torch.distributed), each with its
own replica's timings; the aggregate is all ranks' pairs over the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local, pg = bench.dist_setup()
    dev = torch.device("cpu")
    bench.barrier(pg, dev)
    # rank r took (r + 1) ms per step over 4 steps; 1000 pairs per step on every rank
    value, ms = bench.aggregate(pg, dev, [float(r + 1)] * 4, 1000, 4)
    out.put((r, w, value, ms))
    pg.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, value, ms in res:
        assert w == 2
        # slowest rank: 4 steps x 2 ms = 8 ms; pairs: 2 ranks x 4 x 1000
        assert abs(ms - 2.0) < 1e-12
        assert abs(value - 8000 / 8e-3) < 1e-6
