"""GPU test of bie_apply_static, the operator application that allocates no
device memory.

Some callers of this library may not call cudaMalloc: code embedded in a
host application whose memory manager owns the device heap and forbids other
allocations.  For them the
library keeps the per-call scratch of one operator application in a static
device array.  Here the entry point is called through the C ABI twice in a
row (the array keeps the previous call's contents) and each result is
compared with bie_apply's single-precision-pair application of the same
density, within the tolerance of the mixed-precision apply tests.
"""
import numpy as np
import pytest

from paper_1912_04501_gb300 import workloads

pytestmark = pytest.mark.gpu

bie = pytest.importorskip("paper_1912_04501_gb300.bie")
torch = pytest.importorskip("torch")

MIXED_TOL = 2e-5  # relative max-norm tolerance of the mixed-precision apply tests


@pytest.mark.parametrize("which", ["config2", "two_ellipses_close"])
def test_apply_static_matches_apply(which):
    cell = workloads.config2() if which == "config2" else workloads.two_ellipses(2e-3, 256)
    ctx = bie.Context(cell, precision=bie.BIE_MIXED)
    rng = np.random.default_rng(11)
    for _ in range(2):
        sigma = rng.standard_normal(2 * ctx.N)
        ref = ctx.apply(sigma, precision=bie.BIE_MIXED)
        d_sigma = torch.tensor(sigma, dtype=torch.float64, device="cuda")
        d_out = torch.full_like(d_sigma, float("nan"))
        torch.cuda.synchronize()
        ctx.apply_static(d_sigma, d_out)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() / np.abs(ref).max() < MIXED_TOL
        # same kernels in the same order: the results agree bit for bit
        assert np.array_equal(got, ref)
    ctx.close()


def test_apply_static_rejects_too_many_nodes():
    cell = workloads.small_cell(n_bodies=3, nodes=4096, seed=1)  # 12288 nodes > 8192
    ctx = bie.Context(cell, precision=bie.BIE_MIXED)
    d = torch.zeros(2 * ctx.N, dtype=torch.float64, device="cuda")
    with pytest.raises(bie.BieError) as e:
        ctx.apply_static(d, torch.empty_like(d))
    assert e.value.code == bie.BIE_EINVAL
    assert "8192" in str(e.value)
    ctx.close()


def test_apply_static_rejects_too_much_scratch():
    """A batch of many small cells stays under the node limit but needs more
    scratch than the array holds: the wall-discrepancy partials and proxy
    strengths grow with the number of cells, not with the nodes."""
    cells = []
    for k in range(400):  # 400 cells x 16 nodes = 6400 nodes <= 8192
        cells.append(dict(e1=[1.0, 0.0], e2=[0.0, 1.0], centre=[0.5, 0.5], mu=1.0, gamma=1.0,
                          bodies=[dict(a=0.1, b=0.05, xc=[0.5, 0.5], theta=0.01 * k, n=16)],
                          solver=dict(n_proxy=48, proxy_radius=1.5, n_coll=24, gmres_tol=1e-10)))
    ctx = bie.Context(cells, precision=bie.BIE_MIXED)
    assert ctx.N <= 8192
    d = torch.zeros(2 * ctx.N, dtype=torch.float64, device="cuda")
    with pytest.raises(bie.BieError) as e:
        ctx.apply_static(d, torch.empty_like(d))
    assert e.value.code == bie.BIE_EINVAL
    assert "bytes of scratch" in str(e.value) and str(4 << 20) in str(e.value)
    ctx.close()


def test_apply_static_checks_tensor_sizes():
    cell = workloads.small_cell(n_bodies=2, nodes=64, seed=3)
    ctx = bie.Context(cell, precision=bie.BIE_MIXED)
    d = torch.zeros(2 * ctx.N, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ctx.apply_static(d[:-2], torch.empty_like(d))
    with pytest.raises(ValueError):
        ctx.apply_static(d, d)
    ctx.close()
