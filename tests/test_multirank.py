"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
models, whole-job throughput = all ranks' units over the slowest rank's time
(weak scaling, no data-path collective)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    value, t = bench.job_throughput(local_ms, 400 * 5, dist)
    pool = bench.rank_pool(rank, 8, 2)
    dist.barrier()
    q.put((rank, value, t, pool))
    dist.destroy_process_group()


def test_two_rank_throughput_and_disjoint_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, v, t, pool = q.get(timeout=120)
        res[r] = (v, t, pool)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank reports the same job figure: 2 x 2000 units over 20 ms
    for r in range(world):
        v, t, _ = res[r]
        assert t == pytest.approx(20.0)
        assert v == pytest.approx(2 * 2000 / 0.020)
    # the ranks' parameter sets differ (each rank does its own share)
    assert not np.allclose(res[0][2], res[1][2])


def test_single_rank_throughput():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    v, t = bench.job_throughput(8.0, 1000)
    assert t == 8.0 and v == pytest.approx(1000 / 0.008)
