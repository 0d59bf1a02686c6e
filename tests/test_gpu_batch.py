"""GPU tests of batched contexts (bie_init_batch): several independent unit
cells in one context, one launch per kernel for all of them.

Every cell of a batch must give what a context of its own gives:
* FP64 and double-float operators: relative 1e-12.  Both contexts build the
  same proxy fits and wall discrepancies bit for bit; only the near-sum
  source splits (sized over the whole batch) change the rounding order.
* Single-precision-pair operator: 2e-5, the mixed tolerance of the parity
  tests (the splits change the FP32 rounding).
* Solutions: 1e-9 relative; v, omega, mu_eff: 1e-9 absolute.
One small batch is also checked against the oracle directly (1e-10, the FP64
parity tolerance).
"""
import numpy as np
import pytest

from paper_1912_04501_gb300 import workloads
from tests.conftest import oracle_operator

pytestmark = pytest.mark.gpu

bie = pytest.importorskip("paper_1912_04501_gb300.bie")

SOLVER = dict(n_proxy=32, proxy_radius=1.5, n_coll=16, gmres_tol=1e-10)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


def _batch():
    """Four cells of different sizes, lattices, viscosities and shear rates:
    one body; three ragged bodies on a skew lattice; five bodies of 136 nodes;
    the close pair of Sec. 8 Example 1 (gap 2e-3)."""
    cells = [workloads.config1(),
             workloads.small_cell(n_bodies=3, nodes=(lambda a, b: 50 + int(400 * a)), seed=5, e2=(0.3, 1.0)),
             workloads.small_cell(n_bodies=5, nodes=136, seed=7, phi=0.25, e2=(-0.2, 1.0)),
             workloads.two_ellipses(2e-3, 160, mu=2.0, gamma=0.5)]
    cells[1]["mu"], cells[1]["gamma"] = 0.7, 1.3
    for c in cells:
        c["solver"] = dict(SOLVER)
        for bd in c["bodies"]:
            bd["n"] += bd["n"] % 2
    return cells


def _slices(ctx):
    no = ctx.node_offsets
    return [slice(2 * no[k], 2 * no[k + 1]) for k in range(ctx.n_cells)]


@pytest.fixture(scope="module")
def batch():
    cells = _batch()
    ctx = bie.Context(cells, precision=bie.BIE_FP64, gmres_tol=1e-12)
    singles = [bie.Context(c, precision=bie.BIE_FP64, gmres_tol=1e-12) for c in cells]
    yield cells, ctx, singles
    ctx.close()
    for s in singles:
        s.close()


def test_layout(batch):
    cells, ctx, singles = batch
    assert ctx.n_cells == len(cells)
    assert ctx.N == sum(s.N for s in singles)
    assert list(np.diff(ctx.node_offsets)) == [s.N for s in singles]
    assert list(np.diff(ctx.body_offsets)) == [len(c["bodies"]) for c in cells]
    x, n, w, k = ctx.nodes()
    for sl, s in zip(_slices(ctx), singles):
        xs, ns, ws, ks = s.nodes()
        half = slice(sl.start // 2, sl.stop // 2)
        assert np.array_equal(x[half], xs) and np.array_equal(w[half], ws)


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-12), ("DF64", 1e-12), ("MIXED", 2e-5)])
def test_apply_matches_single_contexts(batch, prec, tol):
    cells, ctx, singles = batch
    p = getattr(bie, "BIE_" + prec)
    sigma = np.random.default_rng(3).standard_normal(2 * ctx.N)
    y = ctx.apply(sigma, precision=p)
    for sl, s in zip(_slices(ctx), singles):
        assert _rel(y[sl], s.apply(sigma[sl], precision=p)) < tol


def test_rhs_per_cell(batch):
    cells, ctx, singles = batch
    b = ctx.rhs()
    for sl, s in zip(_slices(ctx), singles):
        assert np.array_equal(b[sl], s.rhs())


def test_apply_matches_oracle(batch):
    cells, ctx, singles = batch
    sigma = np.random.default_rng(4).standard_normal(2 * ctx.N)
    y = ctx.apply(sigma, precision=bie.BIE_FP64)
    for sl, c in zip(_slices(ctx), cells):
        ref = oracle_operator(c).apply(sigma[sl].reshape(-1, 2)).ravel()
        assert _rel(y[sl], ref) < 1e-10


def test_solve_and_velocities_match_single(batch):
    cells, ctx, singles = batch
    sig, info = ctx.solve()
    ci = ctx.cell_info()
    v, om, mu = ctx.velocities(sig)
    assert info["rel_residual"] <= 1e-12
    for k, (sl, s) in enumerate(zip(_slices(ctx), singles)):
        ss, si = s.solve()
        assert _rel(sig[sl], ss) < 1e-9
        assert ci[k]["rel_residual"] <= 1e-12 and ci[k]["iterations"] >= 1
        vs, oms, mus = s.velocities(ss)
        bo = slice(ctx.body_offsets[k], ctx.body_offsets[k + 1])
        np.testing.assert_allclose(v[bo], vs, atol=1e-9)
        np.testing.assert_allclose(om[bo], oms, atol=1e-9)
        assert abs(mu[k] - mus) < 1e-9
    # lockstep GMRES: the batch took as many sweeps as its slowest cell
    assert info["iterations"] >= max(c["iterations"] for c in ci)


def test_zero_shear_cell_has_zero_density():
    """A cell with gamma = 0 has right-hand side 0 and solution 0; the other
    cells of the batch are unaffected."""
    cells = _batch()[:3]
    cells[1]["gamma"] = 0.0
    ctx = bie.Context(cells, precision=bie.BIE_MIXED)
    sig, info = ctx.solve()
    sl = _slices(ctx)
    assert np.all(sig[sl[1]] == 0.0)
    one = bie.Context(cells[2], precision=bie.BIE_MIXED)
    ref, _ = one.solve()
    assert _rel(sig[sl[2]], ref) < 1e-9
    ci = ctx.cell_info()
    assert ci[1]["iterations"] == 0 and ci[0]["iterations"] > 0
    ctx.close()
    one.close()


def test_mixed_solve_residual_per_cell():
    cells = _batch()
    ctx = bie.Context(cells, precision=bie.BIE_MIXED)
    sig, info = ctx.solve()
    b = ctx.rhs()
    r = b - ctx.apply(sig, precision=bie.BIE_FP64)
    for sl in _slices(ctx):
        assert np.linalg.norm(r[sl]) / np.linalg.norm(b[sl]) <= 1e-10
    ctx.close()


def test_step_matches_single_contexts():
    cells = _batch()[:3]
    dt, n = 2e-3, 2
    ctx = bie.Context(cells, precision=bie.BIE_FP64, gmres_tol=1e-12)
    mu, _ = ctx.step(dt, n)
    st = ctx.get_state()
    assert mu.shape == (n, len(cells)) and st["e2"].shape == (len(cells), 2)
    for k, c in enumerate(cells):
        s = bie.Context(c, precision=bie.BIE_FP64, gmres_tol=1e-12)
        mus, _ = s.step(dt, n)
        ss = s.get_state()
        bo = slice(ctx.body_offsets[k], ctx.body_offsets[k + 1])
        np.testing.assert_allclose(mu[:, k], mus, atol=1e-9)
        np.testing.assert_allclose(st["xc"][bo], ss["xc"], atol=1e-9)
        np.testing.assert_allclose(st["theta"][bo], ss["theta"], atol=1e-9)
        assert np.array_equal(st["e2"][k], ss["e2"])
        s.close()
    ctx.close()


def test_checkpoint_resume_bitwise():
    cells = _batch()[:3]
    a = bie.Context(cells, precision=bie.BIE_MIXED)
    a.step(1e-3, 4)  # the recycled directions (densities, second-sweep correction) are in use
    st = a.get_state()
    assert st["sigma_prev2"] is not None and st["d2"] is not None
    mu_a, _ = a.step(1e-3, 1)
    after_a = a.get_state()
    b = bie.Context(cells, precision=bie.BIE_MIXED)
    b.set_state(st["t"], st["e2"], st["xc"], st["theta"], st["sigma"], st["sigma_prev2"], st["dt_prev"],
                st["d2"])
    mu_b, _ = b.step(1e-3, 1)
    after_b = b.get_state()
    assert np.array_equal(mu_a, mu_b)
    assert np.array_equal(after_a["xc"], after_b["xc"]) and np.array_equal(after_a["sigma"], after_b["sigma"])
    a.close()
    b.close()


def test_min_gap_stops_step():
    """opts.min_gap: a step that leaves two bodies closer than min_gap
    returns BIE_ECOLLIDE (the close pair of Example 1 starts 2e-3 apart)."""
    cell = workloads.two_ellipses(2e-3, 160)
    ctx = bie.Context(cell, precision=bie.BIE_MIXED, min_gap=1e-2)
    with pytest.raises(bie.BieError) as e:
        ctx.step(1e-4, 1)
    assert e.value.code == bie.BIE_ECOLLIDE
    ctx.close()
    ok = bie.Context(cell, precision=bie.BIE_MIXED, min_gap=1e-4)
    ok.step(1e-4, 1)
    ok.close()


def test_apply_static_batch():
    """The allocation-free application serves batches too (same kernels,
    same order: bit for bit the mixed application)."""
    torch = pytest.importorskip("torch")
    cells = _batch()
    ctx = bie.Context(cells, precision=bie.BIE_MIXED)
    assert ctx.N <= 8192
    sigma = np.random.default_rng(8).standard_normal(2 * ctx.N)
    ref = ctx.apply(sigma, precision=bie.BIE_MIXED)
    ds = torch.tensor(sigma, dtype=torch.float64, device="cuda")
    do = torch.full_like(ds, float("nan"))
    torch.cuda.synchronize()
    ctx.apply_static(ds, do)
    torch.cuda.synchronize()
    assert np.array_equal(do.cpu().numpy(), ref)
    ctx.close()


def test_config4_full_batch():
    """The 64-cell ensemble (5-50 bodies per cell, ~300k nodes) in one
    context: two cells against contexts of their own, then the batched mixed
    solve meets the FP64 tolerance in every cell."""
    cells = workloads.config4()
    ctx = bie.Context(cells, precision=bie.BIE_MIXED)
    sigma = np.random.default_rng(9).standard_normal(2 * ctx.N)
    sl = _slices(ctx)
    y64 = ctx.apply(sigma, precision=bie.BIE_FP64)
    y32 = ctx.apply(sigma, precision=bie.BIE_MIXED)
    for k in (0, 37):
        s = bie.Context(cells[k], precision=bie.BIE_MIXED)
        assert _rel(y64[sl[k]], s.apply(sigma[sl[k]], precision=bie.BIE_FP64)) < 1e-12
        assert _rel(y32[sl[k]], s.apply(sigma[sl[k]], precision=bie.BIE_MIXED)) < 2e-5
        s.close()
    sig, info = ctx.solve()
    b = ctx.rhs()
    r = b - ctx.apply(sig, precision=bie.BIE_FP64)
    for s_ in sl:
        assert np.linalg.norm(r[s_]) / np.linalg.norm(b[s_]) <= 1e-10
    ci = ctx.cell_info()
    assert max(c["rel_residual"] for c in ci) <= 1e-10
    ctx.close()
