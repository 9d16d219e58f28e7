"""World-size-2 check of the weak-scaling bookkeeping of bench.py on CPU (gloo): each rank
times its own independent parameter point; the job value is the points of all ranks over
the slowest rank's step time.  No data-path collective is involved."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import numpy as np
    import bench
    import seeded as S

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    value, ms_max = bench.weak_scaling_value(1000, 10.0 * (rank + 1), dist)
    # each rank seeds its own parameter point (bench uses seed 1000 + rank)
    g = dict(n1=5, n2w=3, n2v=3, n3w=3, n3v=3)
    k1 = S.seeded_vertex(g, 1.0, seed=1000 + rank)[0][0]
    dist.destroy_process_group()
    q.put((rank, value, ms_max, np.asarray(k1)))


def test_weak_scaling_two_ranks_gloo():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda t: t[0])
    for rank, value, ms_max, _ in res:
        assert ms_max == pytest.approx(20.0)
        assert value == pytest.approx(2 * 1000 / 20e-3)
    assert not (res[0][3] == res[1][3]).all()


def test_single_rank_value():
    sys.path.insert(0, ROOT)
    import bench

    v, ms = bench.weak_scaling_value(500, 5.0)
    assert ms == 5.0 and v == pytest.approx(500 / 5e-3)
