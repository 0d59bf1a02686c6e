"""GPU parity of the paper's own periodizer (opts.n_images = 4; Def. Gnear,
Sec. 6.1 remark after Eq. W, Sec. 6.2) against the oracle's OperatorUtilde:
each node's four images inside the doubled cell, proxies on the doubled
cell's walls, the periodic sums taken at each node's translate inside U.

Tolerances as in test_gpu_parity.py: FP64 and double-float operators 1e-10
relative (same sums in another order, each side factoring its own proxy
matrix); single-precision pairs 2e-5 (5e-5 at sampled targets of large
cells); solutions to 1e-12 on both sides compared at 1e-9.
"""
import numpy as np
import pytest

from oracle import bie as obie
from oracle import periodic
from paper_1912_04501_gb300 import workloads
from tests.conftest import oracle_suspension

pytestmark = pytest.mark.gpu

bie = pytest.importorskip("paper_1912_04501_gb300.bie")

M_BOX, M_COLL = 128, 32


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


def _cell(kind):
    """Skewed cells: one body across the right wall (nodes outside U), one
    straddling the quadrant lines at the centre; 'close' adds a body 2e-3
    from the first (close-evaluation pairs); 'ragged' uses uneven node
    counts that span several target tiles."""
    e1, e2, c = np.array([1.0, 0.0]), np.array([0.3, 1.0]), np.array([0.5, 0.5])

    def at(s, t):
        return (c + s * e1 + t * e2).tolist()

    n = {"crossing": (128, 128, 128), "close": (160, 128, 96, 96), "ragged": (302, 170, 522)}[kind]
    bodies = [dict(a=0.12, b=0.06, xc=at(-0.18, 0.16), theta=0.4, n=n[0]),
              dict(a=0.10, b=0.07, xc=at(0.45, -0.15), theta=2.0, n=n[1]),
              dict(a=0.09, b=0.05, xc=at(0.02, -0.02), theta=1.1, n=n[2])]
    if kind == "close":
        up = np.array([-np.sin(0.4), np.cos(0.4)])
        bodies.append(dict(a=0.05, b=0.03, xc=(np.array(bodies[0]["xc"]) + (0.06 + 0.03 + 2e-3) * up).tolist(),
                           theta=0.4, n=n[3]))
    return dict(e1=e1.tolist(), e2=e2.tolist(), centre=c.tolist(), mu=1.0, gamma=1.0, bodies=bodies,
                solver=dict(n_proxy=M_BOX, proxy_radius=1.5, n_coll=M_COLL))


@pytest.fixture(scope="module", params=["crossing", "close", "ragged"])
def pair(request):
    cell = _cell(request.param)
    ctx = bie.Context(cell, precision=bie.BIE_FP64, gmres_tol=1e-12, n_images=4)
    ou = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=M_BOX, n_coll=M_COLL)
    yield request.param, cell, ctx, ou
    ctx.close()


def test_utilde_cells_exercise_the_wrap(pair):
    kind, cell, ctx, ou = pair
    st = periodic.lattice_coords(ou.s.e1, ou.s.e2, ou.s.centre, ou.s.x)
    assert (st[:, 0] >= 0.5).sum() > 5  # nodes evaluated at their translates
    m0 = ou.imgmn[:, 0, 0]
    assert (m0 == -1).any() and (m0 == 0).any()  # both image columns in use
    if kind == "close":
        assert ctx.close_info()[0] > 0 and len(ou.close.pairs) > 0


def test_utilde_apply_fp64_df64_mixed(pair):
    kind, cell, ctx, ou = pair
    rng = np.random.default_rng(21)
    sigma = rng.standard_normal(2 * ctx.N)
    ref = ou.apply(sigma.reshape(-1, 2)).ravel()
    assert _rel(ctx.apply(sigma, precision=bie.BIE_FP64), ref) < 1e-10
    assert _rel(ctx.apply(sigma, precision=bie.BIE_DF64), ref) < 1e-10
    assert _rel(ctx.apply(sigma, precision=bie.BIE_MIXED), ref) < 2e-5


def test_utilde_with_the_papers_close_rule():
    """The doubled cell with the close-evaluation blocks by the paper's
    barycentric rule (opts.close_rule = 1) against the oracle's doubled cell
    with the same rule, on a random density: FP64 and double-float 1e-10,
    mixed 2e-5."""
    cell = _cell("close")
    ctx = bie.Context(cell, precision=bie.BIE_FP64, n_images=4, close_rule=1)
    ou = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=M_BOX, n_coll=M_COLL, close_rule="barycentric")
    assert ctx.close_info()[0] > 0 and len(ou.close.pairs) > 0
    sigma = np.random.default_rng(22).standard_normal(2 * ctx.N)
    ref = ou.apply(sigma.reshape(-1, 2)).ravel()
    assert _rel(ctx.apply(sigma, precision=bie.BIE_FP64), ref) < 1e-10
    assert _rel(ctx.apply(sigma, precision=bie.BIE_DF64), ref) < 1e-10
    assert _rel(ctx.apply(sigma, precision=bie.BIE_MIXED), ref) < 2e-5
    ctx.close()


def test_utilde_differs_from_3x3_operator(pair):
    """The two periodizers define the same periodic operator only up to the
    pressure constant: the applications themselves differ (by far more than
    the parity tolerance), so the tests above do pin the doubled cell."""
    kind, cell, ctx, ou = pair
    c9 = bie.Context(cell, precision=bie.BIE_FP64, n_proxy=48, n_coll=24)
    sigma = np.random.default_rng(22).standard_normal(2 * ctx.N)
    a = ctx.apply(sigma, precision=bie.BIE_FP64)
    b = c9.apply(sigma, precision=bie.BIE_FP64)
    assert _rel(a, b) > 1e-6
    c9.close()


def test_utilde_solve_and_velocities(pair):
    kind, cell, ctx, ou = pair
    sig, info = ctx.solve()
    assert info["rel_residual"] <= 1e-12
    ref, _, _ = obie.solve(ou, tol=1e-12)
    assert _rel(sig, ref.ravel()) < 1e-9
    v, om, mu = ctx.velocities(sig)
    v_ref, om_ref = ou.body_velocities(ref)
    np.testing.assert_allclose(v, v_ref, atol=1e-9)
    np.testing.assert_allclose(om, om_ref, atol=1e-9)
    assert abs(mu - ou.mu_eff(ref)) < 1e-9


def test_utilde_mixed_solve():
    cell = _cell("close")
    ctx = bie.Context(cell, precision=bie.BIE_MIXED, gmres_tol=1e-12, n_images=4)
    sig, info = ctx.solve()
    assert info["rel_residual"] <= 1e-12 and info["applies32"] > info["applies64"]
    ou = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=M_BOX, n_coll=M_COLL)
    ref, _, _ = obie.solve(ou, tol=1e-12)
    assert _rel(sig, ref.ravel()) < 1e-9
    ctx.close()


def test_utilde_steps_match_oracle():
    """Three forward-Euler steps (Sec. 7) of the crossing cell on a shearing
    lattice with the doubled-cell periodizer, against the oracle's Euler
    steps with OperatorUtilde."""
    cell = _cell("crossing")
    dt = 0.02
    ctx = bie.Context(cell, precision=bie.BIE_FP64, gmres_tol=1e-12, n_images=4)
    s = oracle_suspension(cell)
    t = 0.0
    mus_ref = []
    for _ in range(3):
        s, t, out = obie.euler_step(s, cell["e2"], t, dt, dict(n_proxy=M_BOX, n_coll=M_COLL), tol=1e-12,
                                    operator=obie.OperatorUtilde)
        mus_ref.append(out["mu_eff"])
    mus, info = ctx.step(dt, 3)
    st = ctx.get_state()
    np.testing.assert_allclose(mus, mus_ref, atol=1e-9)
    np.testing.assert_allclose(st["xc"], s.xc, atol=1e-10)
    np.testing.assert_allclose(st["theta"], [b["theta"] for b in s.bodies], atol=1e-10)
    np.testing.assert_allclose(st["e2"], s.e2, atol=1e-15)
    ctx.close()


def test_utilde_full_size_config5_sampled():
    """The 400-ellipse cell (102400 nodes) with the doubled cell: FP64,
    double-float and mixed applications at sampled targets against the
    oracle evaluated there alone, and the mixed solve's FP64 residual."""
    cell = workloads.config5()
    ctx = bie.Context(cell, precision=bie.BIE_MIXED, n_images=4, n_proxy=M_BOX, n_coll=M_COLL)
    rng = np.random.default_rng(55)
    idx = np.sort(rng.choice(ctx.N, 16, replace=False))
    ou = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=M_BOX, n_coll=M_COLL,
                             close_targets=np.unique(np.concatenate([[0], idx])))
    sigma = rng.standard_normal(2 * ctx.N)
    ref = ou.apply(sigma.reshape(-1, 2), targets=idx)
    for prec, tol in ((bie.BIE_FP64, 1e-10), (bie.BIE_DF64, 1e-10), (bie.BIE_MIXED, 5e-5)):
        y = ctx.apply(sigma, precision=prec).reshape(-1, 2)[idx]
        assert _rel(y, ref) < tol, (prec, _rel(y, ref))
    sig, info = ctx.solve()
    b = ctx.rhs()
    r = b - ctx.apply(sig, precision=bie.BIE_FP64)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    ctx.close()


def test_utilde_rejects_a_body_too_large():
    """A body wider than half a cell (lattice coordinates -0.1 .. 0.5, so its
    nodes left of the centre line lack the image one cell to the left) with
    a small body 2e-3 from that image's tip: the close pair would see a
    partial body image, and both the oracle and the context refuse the
    geometry."""
    cell = dict(e1=[1.0, 0.0], e2=[0.0, 1.0], centre=[0.5, 0.5], mu=1.0, gamma=1.0,
                bodies=[dict(a=0.3, b=0.04, xc=[0.7, 0.5], theta=0.0, n=256),
                        dict(a=0.03, b=0.03, xc=[0.03 + 2e-3, 0.5], theta=0.0, n=64)],
                solver=dict(n_proxy=M_BOX, proxy_radius=1.5, n_coll=M_COLL))
    with pytest.raises(ValueError):
        obie.OperatorUtilde(oracle_suspension(cell), n_proxy=M_BOX, n_coll=M_COLL)
    with pytest.raises(bie.BieError) as e:
        bie.Context(cell, precision=bie.BIE_FP64, n_images=4)
    assert e.value.code == bie.BIE_EINVAL


@pytest.mark.parametrize("crossing", [False, True])
def test_utilde_contour_mu_eff(crossing):
    """Sec. 6.4 (Eq. contourdef) on the GPU: against the oracle's contour
    formula on the same density (same sums in another order: 1e-12), and
    against the particle-stress average (agreement to discretisation
    accuracy); with a body across the bottom wall D, Eq. (mueff) on D itself
    is far off while the contour formula still holds.  (The 1e-10 bar is
    that of every FP64 comparison with the oracle: each side fits its own
    proxy strengths, whose Tikhonov fit carries rounding of Q into the
    correction at ~1e-11.)"""
    e1, e2, c = np.array([1.0, 0.0]), np.array([0.3, 1.0]), np.array([0.5, 0.5])

    def at(s, t):
        return (c + s * e1 + t * e2).tolist()

    bodies = [dict(a=0.12, b=0.06, xc=at(-0.18, 0.16), theta=0.4, n=128)]
    if crossing:
        bodies.append(dict(a=0.10, b=0.07, xc=at(0.17, -0.46), theta=0.3, n=160))
    else:
        bodies += [dict(a=0.10, b=0.07, xc=at(0.17, -0.15), theta=2.0, n=128),
                   dict(a=0.09, b=0.05, xc=at(0.02, -0.02), theta=1.1, n=128)]
    cell = dict(e1=e1.tolist(), e2=e2.tolist(), centre=c.tolist(), mu=1.0, gamma=1.0, bodies=bodies,
                solver=dict(n_proxy=M_BOX, proxy_radius=1.5, n_coll=M_COLL))
    ctx = bie.Context(cell, precision=bie.BIE_FP64, gmres_tol=1e-12, n_images=4)
    sig, info = ctx.solve()
    ou = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=M_BOX, n_coll=M_COLL)
    ref = ou.mu_eff_contour(sig.reshape(-1, 2))
    got = ctx.mu_eff_contour(sig)
    assert abs(got - ref) < 1e-10 * abs(ref)
    _, _, mu_ps = ctx.velocities(sig)
    assert abs(got - mu_ps) < 1e-9
    if crossing:
        from tests.conftest import oracle_operator
        wall = oracle_operator(cell, use_close=False).mu_eff_wall(sig.reshape(-1, 2))
        assert abs(wall - got) > 1e-2
    ctx.close()


def test_contour_mu_eff_needs_the_doubled_cell():
    cell = _cell("crossing")
    ctx = bie.Context(cell, precision=bie.BIE_FP64)
    with pytest.raises(bie.BieError) as e:
        ctx.mu_eff_contour(np.zeros(2 * ctx.N))
    assert e.value.code == bie.BIE_EINVAL
    ctx.close()
