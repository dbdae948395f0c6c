"""N > 1 path of bench.py on CPU: replicas with no data-path collective; the
timing reduction takes the slowest rank and the value counts every rank's
solves (world_size 2, gloo, 127.0.0.1)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 1.5 + rank          # rank 1 is slower
        tmax = bench.max_over_ranks(mine, dist, "cpu")
        out[rank] = (tmax, bench.job_throughput(tmax, 4, world))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.5, 2 * 4 / 2.5)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), dict(eps=0.6, mass=0.005, steps=1, warmup=0, gpus=2))()
    assert bench.run_reference(args, (4, 4, 4, 4)) is None
    assert capsys.readouterr().out == ""
