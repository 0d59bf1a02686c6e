"""Whole-job aggregation of bench.py over ranks, as two gloo ranks on the
CPU: the slowest rank's time, and the units summed over independent
replicas or (the multi-GPU benchmark, which shards one cell by target) those
of the one shared problem; and the reference arm works on rank 0 only.  The
sharded solve's exchange itself is tested in test_shard_cpu.py."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, ms = bench.whole_job(100.0 * (rank + 1), 10.0 + 5.0 * rank, dist, "cpu")
    shared = bench.whole_job(300.0, 10.0 + 5.0 * rank, dist, "cpu", shared=True)
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = (units, ms, shared)


def test_whole_job_over_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == (300.0, 15.0, (300.0, 15.0))


def test_single_process_whole_job():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(7, 3.5, None, "cpu") == (7.0, 3.5)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(A(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""
