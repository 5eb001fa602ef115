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


def test_reference_arm_is_bounded_and_complete():
    """bench.py --impl reference (the FP64 oracle as the reference arm) ends
    within its time budgets (timed steps and warm-up) whatever K and W are,
    and prints one JSON line with the contract's keys, the steps it actually
    warmed and timed, and the ones requested."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, GBK_REFERENCE_BUDGET_S="1", GBK_REFERENCE_WARM_BUDGET_S="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2000",
                        "--warmup", "20"], capture_output=True, text=True, timeout=600, env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("{")][-1]
    d = json.loads(line)
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    assert d["steps_requested"] == 2000 and d["warmup_requested"] == 20 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
