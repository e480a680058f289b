"""The N > 1 path of bench.py (independent replicas, one rank per GPU) on the
CPU: two gloo ranks on 127.0.0.1 agree on the slowest rank's time and rank 0
reports the whole job's rate.  No GPU needed."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    assert bench.dist_env() == (ws, rank, rank)
    bench.barrier(ws)
    elapsed = [100.0, 125.0][rank]  # ms: rank 1 is the slower one
    value, t_max = bench.whole_job_rate(1000, 50, elapsed, ws)
    q.put((rank, value, t_max))
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, t_max in out:
        assert t_max == 125.0
        # 2 ranks x 1000 cells x 50 steps in 0.125 s
        assert value == pytest.approx(2 * 1000 * 50 / 0.125 / 1e6)
