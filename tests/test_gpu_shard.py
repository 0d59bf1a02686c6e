"""GPU test of the target partition (bie_set_partition), emulating two
processes in one: context A owns the first bodies, context B the others, and
A's exchange fills B's rows from B's own partitioned application of the same
density.  The result must equal the unpartitioned application bit for bit
(the near-sum splits are those of the whole cell, so every owned target's
partial sums are unchanged), in all three precisions.  The collective
itself (an all-gather of the owned slices) and the replicated GMRES are
tested over two gloo ranks in test_shard_cpu.py."""
import numpy as np
import pytest

from paper_1912_04501_gb300 import workloads

pytestmark = pytest.mark.gpu

bie = pytest.importorskip("paper_1912_04501_gb300.bie")
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("images", [9, 4])
def test_partitioned_apply_matches_whole(images):
    from paper_1912_04501_gb300 import shard
    cell = workloads.config2()
    kw = dict(n_images=images) if images == 9 else dict(n_images=4, n_proxy=128, n_coll=32)
    full = bie.Context(cell, precision=bie.BIE_FP64, **kw)
    a = bie.Context(cell, precision=bie.BIE_FP64, **kw)
    b = bie.Context(cell, precision=bie.BIE_FP64, **kw)
    bounds, nodes = shard.partition([bd["n"] for bd in cell["bodies"]], 2)
    (_, k), _ = nodes
    sigma = torch.tensor(np.random.default_rng(4).standard_normal(2 * full.N), dtype=torch.float64, device="cuda")
    yb = torch.empty_like(sigma)
    state = {"prec": bie.BIE_FP64, "calls": 0}

    def exch_b(ptr, n2, user):
        return 0

    def exch_a(ptr, n2, user):
        y = torch.as_tensor(shard._DeviceVector(ptr, n2), device="cuda")
        b.apply(sigma, yb, precision=state["prec"])
        y[2 * k:] = yb[2 * k:]
        torch.cuda.synchronize()
        state["calls"] += 1
        return 0

    cb_a, cb_b = shard.EXCHANGE(exch_a), shard.EXCHANGE(exch_b)
    b.set_partition(bounds[1], bounds[2], cb_b)
    a.set_partition(bounds[0], bounds[1], cb_a)
    for prec in (bie.BIE_FP64, bie.BIE_DF64, bie.BIE_MIXED):
        state["prec"] = prec
        ref = torch.empty_like(sigma)
        full.apply(sigma, ref, precision=prec)
        got = torch.full_like(sigma, float("nan"))
        a.apply(sigma, got, precision=prec)
        assert torch.equal(got, ref), prec
    assert state["calls"] == 3
    # switched off again: no exchange, whole result
    a.set_partition(0, a.n_bodies, None)
    got = torch.empty_like(sigma)
    a.apply(sigma, got, precision=bie.BIE_FP64)
    ref = torch.empty_like(sigma)
    full.apply(sigma, ref, precision=bie.BIE_FP64)
    assert torch.equal(got, ref) and state["calls"] == 3
    for c in (a, b, full):
        c.close()


def test_partition_rejects_bad_ranges():
    cell = workloads.small_cell(n_bodies=3, nodes=64, seed=2)
    ctx = bie.Context(cell, precision=bie.BIE_FP64)
    with pytest.raises(bie.BieError):
        ctx.set_partition(2, 1, None)
    with pytest.raises(bie.BieError):
        ctx.set_partition(0, 2, None)  # a proper part needs an exchange
    ctx.close()


def _solve_rank(rank, world, port, out):
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_1912_04501_gb300 import bie as b, shard, workloads as w
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cell = w.small_cell(n_bodies=6, nodes=(lambda a, c: 96 + 2 * int(80 * a)), seed=9, e2=(0.2, 1.0))
    ctx = b.Context(cell, precision=b.BIE_MIXED)
    sh = shard.ShardedSolve(ctx, [bd["n"] for bd in cell["bodies"]], rank, world)
    sig, info = ctx.solve()
    mus, _ = ctx.step(cell.get("dt", 1e-3), 2)
    st = ctx.get_state()
    sh.close()
    ctx.close()
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = (sig, info["iterations"], mus, st["xc"])


def test_sharded_solve_two_processes_one_gpu():
    """Two processes on one GPU solve and step one cell sharded by target,
    exchanging their rows over a gloo process group (host copies): the
    kernels never wait on one another, the exchange is a host collective
    between launches.  Every process ends with the same density, iteration
    count and trajectory, bit for bit equal to the unsharded solve."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_solve_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    cell = workloads.small_cell(n_bodies=6, nodes=(lambda a, c: 96 + 2 * int(80 * a)), seed=9, e2=(0.2, 1.0))
    ref = bie.Context(cell, precision=bie.BIE_MIXED)
    sig, info = ref.solve()
    mus, _ = ref.step(cell.get("dt", 1e-3), 2)
    st = ref.get_state()
    ref.close()
    for r in (0, 1):
        s_r, it_r, mu_r, xc_r = res[r]
        assert np.array_equal(s_r, sig) and it_r == info["iterations"]
        assert np.array_equal(mu_r, mus) and np.array_equal(xc_r, st["xc"])
