"""GPU tests of the error paths: a solve stopped above its tolerance returns
BIE_ENOCONV with the residual reached (the best iterate is still written);
a non-finite right-hand side returns BIE_ENUMERIC; no GPU fault is involved."""
import numpy as np
import pytest

from paper_1912_04501_gb300 import workloads

pytestmark = pytest.mark.gpu

bie = pytest.importorskip("paper_1912_04501_gb300.bie")


def test_stopped_solve_reports_enoconv():
    cell = workloads.small_cell(n_bodies=3, nodes=96, seed=4)
    ctx = bie.Context(cell, precision=bie.BIE_MIXED, max_refine=1, inner_tol=1e-2)
    with pytest.raises(bie.BieError) as e:
        ctx.solve()
    assert e.value.code == bie.BIE_ENOCONV and "relative residual" in str(e.value)
    sigma, info = ctx.solve(allow_noconv=True)
    assert 1e-10 < info["rel_residual"] < 1.0 and np.isfinite(sigma).all()
    b = ctx.rhs()
    r = b - ctx.apply(sigma, precision=bie.BIE_FP64)
    # the returned iterate is the one the residual was reported for
    assert np.linalg.norm(r) / np.linalg.norm(b) == pytest.approx(info["rel_residual"], rel=1e-6)
    ctx.close()


def test_non_finite_rhs_reports_enumeric():
    cell = workloads.config1()
    ctx = bie.Context(cell, precision=bie.BIE_FP64)
    b = ctx.rhs()
    b[5] = np.nan
    with pytest.raises(bie.BieError) as e:
        ctx.solve(rhs=b)
    assert e.value.code == bie.BIE_ENUMERIC
    # the context stays usable
    sigma, info = ctx.solve()
    assert info["rel_residual"] <= 1e-10
    ctx.close()
