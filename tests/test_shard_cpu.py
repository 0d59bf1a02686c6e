"""The target-sharded solve's host logic (paper_1912_04501_gb300.shard) over
two gloo ranks on the CPU, with the FP64 oracle's application at each
rank's own targets standing in for the library's partitioned application:
after the all-gather every rank holds exactly the unsharded result, and a
GMRES whose matrix-vector products go through the exchange gives every rank
the unsharded solution."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cell():
    from paper_1912_04501_gb300 import workloads
    return workloads.small_cell(n_bodies=5, nodes=(lambda a, b: 40 + int(60 * a)), seed=11, e2=(0.2, 1.0))


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from oracle import bie as obie
    from paper_1912_04501_gb300 import shard
    from tests.conftest import oracle_operator
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cell = _cell()
    op = oracle_operator(cell)
    counts = [bd["n"] for bd in cell["bodies"]]
    bounds, nodes = shard.partition(counts, world)
    a, b = nodes[rank]

    def sharded_matvec(v):
        y = torch.zeros(2 * op.s.N, dtype=torch.float64)
        y[2 * a: 2 * b] = torch.from_numpy(op.apply(v.reshape(-1, 2), targets=np.arange(a, b)).ravel())
        return shard.gather_slices(y, nodes, rank).numpy()

    sigma = np.random.default_rng(3).standard_normal(2 * op.s.N)
    y = sharded_matvec(sigma)
    x, it, _ = obie.gmres(sharded_matvec, op.rhs().ravel(), tol=1e-12)
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = (bounds, nodes, y, x, it)


def test_partition_whole_bodies_balanced():
    from paper_1912_04501_gb300 import shard
    counts = [100, 300, 50, 50, 400, 100]
    bounds, nodes = shard.partition(counts, 3)
    assert bounds[0] == 0 and bounds[-1] == len(counts)
    assert all(bounds[r] < bounds[r + 1] for r in range(3))
    assert nodes[0][0] == 0 and nodes[-1][1] == sum(counts)
    assert all(nodes[r][1] == nodes[r + 1][0] for r in range(2))
    sizes = [b - a for a, b in nodes]
    assert max(sizes) <= 500  # the 400-node body bounds the balance
    with pytest.raises(ValueError):
        shard.partition(counts, 7)
    assert shard.partition([5], 1) == ([0, 1], [(0, 5)])


def test_sharded_apply_and_gmres_over_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    import sys
    sys.path.insert(0, ROOT)
    from oracle import bie as obie
    from tests.conftest import oracle_operator
    op = oracle_operator(_cell())
    sigma = np.random.default_rng(3).standard_normal(2 * op.s.N)
    full = op.apply(sigma.reshape(-1, 2)).ravel()
    (b0, n0, y0, x0, it0), (b1, n1, y1, x1, it1) = res[0], res[1]
    assert b0 == b1 and n0 == n1 and n0[0][1] == n0[1][0]
    # every rank holds the same vector, equal to the unsharded application
    assert np.array_equal(y0, y1)
    np.testing.assert_allclose(y0, full, rtol=0, atol=1e-13 * np.abs(full).max())
    # the replicated GMRES agrees on every rank and with the unsharded solve
    assert np.array_equal(x0, x1) and it0 == it1
    xs, _, _ = obie.gmres(op.matvec, op.rhs().ravel(), tol=1e-12)
    np.testing.assert_allclose(x0, xs, atol=1e-11 * np.abs(xs).max())
