"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks.

Each rank advances its own box; the whole-job value divides the sites of all
ranks by the slowest rank's time.  The reference arm runs on rank 0 only.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = [80.0, 120.0][rank]
    value, t_max = bench.whole_job(ms_local, 1000, 10, world, dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, value, t_max, bench.dist_env()))


def test_whole_job_value_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t_max, env in res:
        assert t_max == 120.0
        # 2 ranks x 1000 sites x 10 steps in 0.12 s
        assert abs(value - 2 * 1000 * 10 / 0.12 / 1e6) < 1e-12
        assert env[0] == rank and env[1] == 2


def test_reference_arm_only_on_rank_zero(monkeypatch, capsys):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 3, 3, 2

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
