"""Pins of the oracle's periodizing machinery (Sec. 4.2, Sec. 6.1, Sec. 6.2).

* App. B / Eq. (W): the discrepancy of the near sum, corrected by g0, is
  consistent (W^T g~ = 0) for ANY density, including non-zero net force; and
  W^T Q = 0.  Flipping the wall normal convention breaks this (planted mistake).
* The cancellation form of the discrepancy equals the literal difference of
  3x3 sums (translation invariance, Sec. 6.2 step 2).
* Sec. 6.1 Example 1 (golden setup): the EBVP for a known Stokeslet field
  converges exponentially in the number of proxies.
* The assembled periodic single layer is periodic in velocity and traction
  when the net force is zero, and its traction jumps by F/(2|e2|), F/(2|e1|)
  otherwise (Definition of G_per, Eqs. gperdiscrep1-4, Remark r:notper); by
  the uniqueness theorem this fixes it up to constants.
* A 5x5 near sum with its own correction gives the same traction after the
  pressure-constant fix (G_per does not depend on the near/correction split).
"""
import math
import os

import numpy as np
import pytest

from oracle import geometry, kernels, periodic
from paper_1912_04501_gb300 import workloads
from tests.conftest import oracle_operator, oracle_suspension

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ebvp_example.txt")


def _cell(e2=(0.3, 1.0), seed=0):
    return workloads.small_cell(n_bodies=3, nodes=64, seed=seed, e2=e2)


@pytest.mark.parametrize("e2", [(0.0, 1.0), (0.3, 1.0), (-0.45, 1.0)])
def test_consistency_any_net_force(e2):
    cell = _cell(e2)
    op = oracle_operator(cell)
    s = op.s
    W = periodic.consistency_matrix(s.e1, s.e2, s.centre, op.m)
    rng = np.random.default_rng(3)
    sig = rng.normal(size=(s.N, 2))
    q, F, _ = op.density_moments(sig)
    assert np.abs(F).max() > 1e-2
    _, dt = op.proxy_strengths(q)
    assert np.abs(W @ dt).max() < 1e-12 * max(1.0, np.abs(dt).max())
    assert np.abs(W @ op.Q).max() < 1e-13 * np.abs(op.Q).max()


def test_consistency_fails_with_flipped_wall_normals(monkeypatch):
    """Plant the other normal convention in the oracle: consistency breaks by
    O(F), so the test above really checks the sign."""
    cell = _cell()
    orig = periodic.wall_normals
    monkeypatch.setattr(periodic, "wall_normals", lambda e1, e2: tuple(-v for v in orig(e1, e2)))
    op = oracle_operator(cell)
    s = op.s
    W = periodic.consistency_matrix(s.e1, s.e2, s.centre, op.m)
    sig = np.random.default_rng(3).normal(size=(s.N, 2))
    q, F, _ = op.density_moments(sig)
    _, dt = op.proxy_strengths(q)
    assert np.abs(W[:2] @ dt - 2 * F.sum(0)).max() < 1e-10


def test_discrepancy_cancellation_matches_literal_difference():
    cell = _cell()
    # bodies well inside the cell so the literal difference is not ill-conditioned
    for bd in cell["bodies"]:
        bd["xc"] = [0.5 + 0.25 * (bd["xc"][0] - 0.5), 0.5 + 0.25 * (bd["xc"][1] - 0.5)]
        bd["a"] *= 0.5
        bd["b"] *= 0.5
    s = oracle_suspension(cell)
    q = np.random.default_rng(1).normal(size=(s.N, 2)) * s.w[:, None]
    g_fast = periodic.near_discrepancy(s.e1, s.e2, s.centre, 12, s.x, q, s.mu)
    g_lit = periodic.near_discrepancy_direct(s.e1, s.e2, s.centre, 12, s.x, q, s.mu)
    np.testing.assert_allclose(g_fast, g_lit, atol=1e-12 * np.abs(g_lit).max())


def _read_golden():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        vals[k] = v
    ev = lambda t: eval(t, {"cos": math.cos, "sin": math.sin, "pi": math.pi})
    mu = float(vals["mu"][0])
    y0 = np.array([ev(t) for t in vals["y0"]])
    f0 = np.array([float(t) for t in vals["f0"]])
    cells = {}
    for key in ("cell_square", "cell_skew"):
        v = vals[key]
        cells[key] = (np.array([ev(v[1]), ev(v[2])]), np.array([ev(v[4]), ev(v[5])]),
                      np.array([ev(v[7]), ev(v[8])]))
    return mu, y0, f0, cells, int(vals["grid"][0])


def _ebvp_error(mu, y0, f0, e1, e2, c, M, m, ngrid):
    yp = periodic.proxy_points_box(e1, e2, c, M)
    Q = periodic.proxy_matrix(e1, e2, c, m, yp, mu)
    xl, xd, _, _ = periodic.collocation(e1, e2, c, m)
    nl, nd = periodic.wall_normals(e1, e2)
    v = lambda x: kernels.stokeslet(x - y0, f0[None, :], mu)
    t = lambda x, nu: kernels.traction(x - y0, np.repeat(nu[None], len(x), 0), f0[None, :])
    sp = periodic._split
    d = np.concatenate([sp(v(xl + e1) - v(xl)), sp(t(xl + e1, nl) - t(xl, nl)),
                        sp(v(xd + e2) - v(xd)), sp(t(xd + e2, nd) - t(xd, nd))])
    xi = periodic.proxy_solution_operator(Q) @ d
    s = np.linspace(-0.5, 0.5, ngrid)
    S1, S2 = np.meshgrid(s, s, indexing="ij")
    grid = c + S1.reshape(-1, 1) * e1 + S2.reshape(-1, 1) * e2
    err = periodic.correction_velocity(grid, yp, xi, mu) - v(grid)
    err -= err[0]
    return np.abs(err).max() / np.abs(v(grid)).max()


@pytest.mark.parametrize("key", ["cell_square", "cell_skew"])
def test_ebvp_example_converges(key):
    mu, y0, f0, cells, ngrid = _read_golden()
    e1, e2, c = cells[key]
    errs = [_ebvp_error(mu, y0, f0, e1, e2, c, M, m, ngrid)
            for M, m in [(16, 8), (32, 16), (48, 24), (64, 32)]]
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[1] / errs[0] < 0.1 and errs[2] / errs[1] < 0.1
    assert errs[3] < 1e-7


def _periodic_fields(op, sig):
    s = op.s
    q, _, _ = op.density_moments(sig)
    xi, _ = op.proxy_strengths(q)
    U = lambda x: periodic.near_velocity(x, s.x, q, op.shifts, s.mu) + \
        periodic.correction_velocity(x, op.yp, xi, s.mu)
    T = lambda x, nu: periodic.near_traction(x, np.repeat(nu[None], len(x), 0), s.x, q, op.shifts) + \
        periodic.correction_traction(x, np.repeat(nu[None], len(x), 0), op.yp, xi)
    return U, T, q


@pytest.mark.parametrize("e2", [(0.0, 1.0), (0.3, 1.0)])
def test_periodic_and_force_jump(e2):
    cell = _cell(e2)
    op = oracle_operator(cell, n_proxy=48, n_coll=24)
    s = op.s
    rng = np.random.default_rng(11)
    sig = rng.normal(size=(s.N, 2))
    nl, nd = periodic.wall_normals(s.e1, s.e2)
    sl = rng.uniform(-0.5, 0.5, 15)
    xl = s.centre - 0.5 * s.e1 + sl[:, None] * s.e2
    xd = s.centre - 0.5 * s.e2 + sl[:, None] * s.e1
    # zero net force: remove the mean of q body by body
    sig0 = sig.copy()
    for b in range(len(s.bodies)):
        k = slice(s.offsets[b], s.offsets[b + 1])
        sig0[k] -= (sig0[k] * s.w[k, None]).sum(0) / s.w[k].sum()
    U, T, q = _periodic_fields(op, sig0)
    scale = np.abs(U(xl)).max()
    assert np.abs(U(xl + s.e1) - U(xl)).max() < 3e-8 * max(1, scale)
    assert np.abs(U(xd + s.e2) - U(xd)).max() < 3e-8 * max(1, scale)
    assert np.abs(T(xl + s.e1, nl) - T(xl, nl)).max() < 3e-8 * max(1, np.abs(T(xl, nl)).max())
    # non-zero net force: velocity still periodic, traction jumps by F/(2|e|)
    U, T, q = _periodic_fields(op, sig)
    F = q.sum(0)
    assert np.abs(U(xl + s.e1) - U(xl)).max() < 3e-8 * max(1, np.abs(U(xl)).max())
    jump_lr = T(xl + s.e1, nl) - T(xl, nl)
    jump_du = T(xd + s.e2, nd) - T(xd, nd)
    np.testing.assert_allclose(jump_lr, np.repeat((F / (2 * np.hypot(*s.e2)))[None], 15, 0), atol=3e-8)
    np.testing.assert_allclose(jump_du, np.repeat((F / (2 * np.hypot(*s.e1)))[None], 15, 0), atol=3e-8)


def test_near_split_independence_5x5():
    """G_per is unique up to constants (Thm t:consistency + Lemma l:bvpunique):
    a 5x5 near sum corrected by its own MFS fit gives the same traction as the
    3x3 one once the pressure constant (a multiple of n) is removed."""
    cell = _cell((0.2, 1.0))
    op = oracle_operator(cell, n_proxy=48, n_coll=24, use_close=False)
    s = op.s
    sig = np.random.default_rng(4).normal(size=(s.N, 2))
    T3 = op.traction(sig)
    # 5x5 variant assembled from the same oracle pieces with a wider discrepancy
    shifts5 = [m * s.e1 + n * s.e2 for n in range(-2, 3) for m in range(-2, 3)]
    q, _, _ = op.density_moments(sig)
    T5 = periodic.near_traction(s.x, s.n, s.x, q, shifts5, self_index=np.arange(s.N))
    T5 += kernels.traction_self(s.kappa, s.tau, q)
    xl, xd, _, _ = periodic.collocation(s.e1, s.e2, s.centre, op.m)
    nl, nd = periodic.wall_normals(s.e1, s.e2)
    m = op.m
    nlm, ndm = np.repeat(nl[None], m, 0), np.repeat(nd[None], m, 0)
    # 5x5 discrepancy, computed literally (sources are >= ~1.5 cells from the walls' far images)
    g1 = periodic.near_velocity(xl + s.e1, s.x, q, shifts5, s.mu) - periodic.near_velocity(xl, s.x, q, shifts5, s.mu)
    g2 = periodic.near_traction(xl + s.e1, nlm, s.x, q, shifts5) - periodic.near_traction(xl, nlm, s.x, q, shifts5)
    g3 = periodic.near_velocity(xd + s.e2, s.x, q, shifts5, s.mu) - periodic.near_velocity(xd, s.x, q, shifts5, s.mu)
    g4 = periodic.near_traction(xd + s.e2, ndm, s.x, q, shifts5) - periodic.near_traction(xd, ndm, s.x, q, shifts5)
    sp = periodic._split
    g = np.concatenate([sp(g1), sp(g2), sp(g3), sp(g4)])
    dt = periodic.corrected_discrepancy(g, q.sum(0), s.e1, s.e2, m)
    T5 += periodic.correction_traction(s.x, s.n, op.yp, op.Qp @ dt)
    fix = lambda T: T - (T[0] @ s.n[0]) * s.n
    d = fix(T3) - fix(T5)
    assert np.abs(d).max() < 3e-7 * np.abs(fix(T3)).max()


def test_paper_periodizer_agrees_with_3x3():
    """Reading 1 (3 x 3 images of every body, proxies on a circle) against
    the paper's own periodizer (Def. Gnear: each node's four images inside
    the doubled cell, chosen per node by its lattice coordinates; proxies on
    the doubled cell's walls).  Both define the same periodic Green's
    function up to constants, so on a skewed cell whose bodies straddle the
    quadrant lines (nodes on both sides get different image sets) the
    densities, rotation rates, relative velocities and mu_eff agree to the
    accuracy of the proxy fits (~1e-9), while the absolute velocities differ
    by one constant (the free constant of the periodic Green's function)."""
    from oracle import bie as obie
    e1, e2, c = np.array([1.0, 0.0]), np.array([0.3, 1.0]), np.array([0.5, 0.5])

    def at(s, t):
        return (c + s * e1 + t * e2).tolist()

    cell = dict(e1=e1.tolist(), e2=e2.tolist(), centre=c.tolist(), mu=1.0, gamma=1.0,
                bodies=[dict(a=0.12, b=0.06, xc=at(-0.18, 0.16), theta=0.4, n=128),
                        dict(a=0.10, b=0.07, xc=at(0.17, -0.15), theta=2.0, n=128),
                        dict(a=0.09, b=0.05, xc=at(0.02, -0.02), theta=1.1, n=128)],
                solver=dict(n_proxy=48, proxy_radius=1.5, n_coll=24))
    op = oracle_operator(cell, use_close=False)
    st = np.linalg.solve(np.column_stack([e1, e2]), (op.s.x - c).T).T
    assert np.abs(st).max() < 0.5 and (st[:, 0] < 0).any() and (st[:, 0] > 0).any() and (st[:, 1] < 0).any()
    ou = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=128, n_coll=32)
    s3, _, r3 = obie.solve(op, tol=1e-12)
    su, _, ru = obie.solve(ou, tol=1e-12)
    assert r3 <= 1e-12 and ru <= 1e-12
    v3, w3 = op.body_velocities(s3)
    vu, wu = ou.body_velocities(su)
    assert np.abs(su - s3).max() / np.abs(s3).max() < 1e-8
    assert np.abs(wu - w3).max() < 1e-9
    assert np.abs((vu - vu[0]) - (v3 - v3[0])).max() < 1e-9
    assert abs(ou.mu_eff(su) - op.mu_eff(s3)) < 1e-9
    const = vu - v3
    assert np.abs(const - const[0]).max() < 1e-9 and np.abs(const[0]).max() > 1e-6
    # planted mistake: each node's images taken on the wrong side (shifts
    # m e1 + n e2 negated, so three of the four lie outside the doubled
    # cell).  The wall proxies absorb most of it (any image set plus an exact
    # correction gives the same periodic sum), but the images left just
    # outside U move sigma by ~1.6e-6, far above the 1e-9 agreement
    bad = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=128, n_coll=32)
    bad.img = -bad.img
    sb, _, _ = obie.solve(bad, tol=1e-12)
    assert np.abs(sb - s3).max() / np.abs(s3).max() > 1e-7


def _crossing_cell(n=128, close_pair=False, crossing=True):
    """A skewed cell with one body across the right wall (nodes outside U;
    inside U near that wall if not crossing), one straddling the quadrant
    lines at the centre, and optionally a fourth body a small gap from the
    first (a close-evaluation pair)."""
    e1, e2, c = np.array([1.0, 0.0]), np.array([0.3, 1.0]), np.array([0.5, 0.5])

    def at(s, t):
        return (c + s * e1 + t * e2).tolist()

    bodies = [dict(a=0.12, b=0.06, xc=at(-0.18, 0.16), theta=0.4, n=n),
              dict(a=0.10, b=0.07, xc=at(0.45 if crossing else 0.3, -0.15), theta=2.0, n=n),
              dict(a=0.09, b=0.05, xc=at(0.02, -0.02), theta=1.1, n=n)]
    if close_pair:
        # an ellipse 2e-3 above the first one's top (its semi-axis b = 0.06 at theta = 0.4)
        bodies.append(dict(a=0.05, b=0.03, xc=at(-0.18, 0.16), theta=0.4, n=n))
        th = 0.4
        up = np.array([-np.sin(th), np.cos(th)])
        bodies[-1]["xc"] = (np.array(bodies[0]["xc"]) + (0.06 + 0.03 + 2e-3) * up).tolist()
    return dict(e1=e1.tolist(), e2=e2.tolist(), centre=c.tolist(), mu=1.0, gamma=1.0, bodies=bodies,
                solver=dict(n_proxy=48, proxy_radius=1.5, n_coll=24))


def test_utilde_discrepancy_cancellation_matches_literal():
    """Sec. 6.2 step 2 for the doubled-cell near sum: the cancellation form
    (two far terms per image row of every node) equals the literal
    S_near(R) - S_near(L), S_near(U) - S_near(D) over the expanded image list
    when no body comes near a wall; a wrong column in either term (planted
    here: m0 + 2 instead of m0 + 1) does not."""
    from oracle import bie as obie
    cell = _crossing_cell()
    cell["bodies"] = [cell["bodies"][0], cell["bodies"][2]]  # nothing near a wall
    ou = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=64, n_coll=16, use_close=False)
    s = ou.s
    q = np.random.default_rng(5).normal(size=(s.N, 2)) * s.w[:, None]
    Y, Q, _ = ou._sources(q)
    lit = periodic.near_discrepancy_images(s.e1, s.e2, s.centre, 16, Y, Q, s.mu)
    can = periodic.near_discrepancy_utilde(s.e1, s.e2, s.centre, 16, s.x, q, ou.imgmn, s.mu)
    np.testing.assert_allclose(can, lit, atol=1e-12 * np.abs(lit).max())
    bad = ou.imgmn.copy()
    bad[:, :, 0] += 1
    wrong = periodic.near_discrepancy_utilde(s.e1, s.e2, s.centre, 16, s.x, q, bad, s.mu)
    assert np.abs(wrong - lit).max() > 1e-3 * np.abs(lit).max()


def test_utilde_wrapped_targets_agree_with_3x3():
    """A body across a wall: Sec. 6.2 evaluates the periodic sums at targets
    in U, so the doubled-cell operator takes each outside node at its lattice
    translate inside U.  Against reading 1 (3 x 3 images of every body) the
    densities then agree to ~7e-8 and the rotation rates to ~3e-8 (both
    periodizers' proxy fits are accurate to ~1e-8 near the walls; the two
    traction fields agree to 1e-9 inside U)."""
    from oracle import bie as obie
    cell = _crossing_cell()
    op = oracle_operator(cell, use_close=False)
    st = periodic.lattice_coords(op.s.e1, op.s.e2, op.s.centre, op.s.x)
    assert (st[:, 0] >= 0.5).sum() > 10
    ou = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=128, n_coll=32, use_close=False)
    s3, _, _ = obie.solve(op, tol=1e-12)
    su, _, _ = obie.solve(ou, tol=1e-12)
    v3, w3 = op.body_velocities(s3)
    vu, wu = ou.body_velocities(su)
    assert np.abs(su - s3).max() / np.abs(s3).max() < 2e-7
    assert np.abs(wu - w3).max() < 1e-7
    assert np.abs((vu - vu[0]) - (v3 - v3[0])).max() < 1e-8
    assert abs(ou.mu_eff(su) - op.mu_eff(s3)) < 1e-8


def test_utilde_close_evaluation_agrees_with_3x3():
    """Two bodies 2e-3 apart (well inside each other's close zones): with the
    close-evaluation correction of Sec. 6.3 taken pair for pair in the nodes'
    own frame, the doubled-cell operator agrees with reading 1 to the
    accuracy of the proxy fits; without the correction the density moves by
    far more.  (With a body across a wall as well, the near-contact density,
    ~20x larger than elsewhere, raises the 3 x 3 operator's own periodicity
    error at the nodes outside U to ~2e-7, and the two then agree to ~4e-7.)"""
    from oracle import bie as obie
    cell = _crossing_cell(close_pair=True, crossing=False)
    op = oracle_operator(cell)
    assert len(op.close.pairs) > 20
    ou = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=128, n_coll=32)
    s3, _, _ = obie.solve(op, tol=1e-12)
    su, _, _ = obie.solve(ou, tol=1e-12)
    _, w3 = op.body_velocities(s3)
    _, wu = ou.body_velocities(su)
    assert np.abs(su - s3).max() / np.abs(s3).max() < 2e-7
    assert np.abs(wu - w3).max() < 1e-7
    nc = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=128, n_coll=32, use_close=False)
    sn, _, _ = obie.solve(nc, tol=1e-12)
    assert np.abs(sn - s3).max() / np.abs(s3).max() > 1e-4


def _ewald_stokeslet_velocity(xt, ys, fs, e1, e2, mu, xi, nreal=3, kmax=14):
    """Velocity of periodic point forces with zero total (zero cell-mean
    flow), by Hasimoto's Ewald split of the Stokeslet, written out here as an
    independent classical route: 1/k^4 = phi/k^4 + (1 - phi)/k^4 with
    phi = (1 + k^2/(4 xi^2)) exp(-k^2/(4 xi^2)).  The real-space part of one
    force f is R(r) f with
        R = [(E1(xi^2 r^2)/2 - exp(-xi^2 r^2)) I + exp(-xi^2 r^2) r r^T / r^2] / (4 pi mu)
    (its r -> 0 limit is the Stokeslet (-log r I + r r^T / r^2) / (4 pi mu)
    plus a constant), the Fourier part (I - k k^T / k^2) phi / (mu |U| k^2)
    over the reciprocal lattice without k = 0.  For zero total force the sum
    does not depend on xi."""
    from scipy.special import exp1
    E = np.column_stack([e1, e2])
    area = abs(np.linalg.det(E))
    B = 2 * np.pi * np.linalg.inv(E).T
    u = np.zeros((len(xt), 2))
    for m in range(-nreal, nreal + 1):
        for n in range(-nreal, nreal + 1):
            r = xt[:, None, :] - (ys[None, :, :] + m * e1 + n * e2)
            r2 = (r * r).sum(-1)
            X = xi * xi * r2
            ex = np.exp(-X)
            rf = (r * fs[None, :, :]).sum(-1)
            u += ((0.5 * exp1(X) - ex)[..., None] * fs[None, :, :] + (ex * rf / r2)[..., None] * r).sum(1)
    u /= 4 * np.pi * mu
    for m in range(-kmax, kmax + 1):
        for n in range(-kmax, kmax + 1):
            if m == 0 and n == 0:
                continue
            k = B @ np.array([m, n])
            k2 = k @ k
            phi = (1 + k2 / (4 * xi * xi)) * np.exp(-k2 / (4 * xi * xi))
            P = np.eye(2) - np.outer(k, k) / k2
            ph = np.exp(1j * ((xt[:, None, :] - ys[None, :, :]) @ k))
            u += np.real((ph[..., None] * (fs @ P.T)[None, :, :]).sum(1)) * phi / (mu * area * k2)
    return u


@pytest.mark.parametrize("skew", [0.0, 0.3])
def test_periodic_stokeslet_matches_ewald(skew):
    """The oracle's periodic Green's function (3 x 3 near sum + proxy
    correction, Sec. 6.2) against the Ewald sum above, for five point forces
    of zero total in a square and a skewed cell: equal up to one constant
    velocity (G_per's free constant) to ~1e-9 of the velocity scale.  The
    Ewald sum is itself checked by its independence of the splitting
    parameter.  A near sum without the four diagonal images (planted
    mistake) fails."""
    rng = np.random.default_rng(3 + int(10 * skew))
    e1, e2, c, mu = np.array([1.0, 0.0]), np.array([skew, 1.0]), np.array([0.5, 0.5]), 1.3
    E = np.column_stack([e1, e2])
    ys = c + rng.uniform(-0.4, 0.4, (5, 2)) @ E.T
    fs = rng.standard_normal((5, 2))
    fs -= fs.mean(0)
    xt = c + rng.uniform(-0.45, 0.45, (7, 2)) @ E.T
    u_a = _ewald_stokeslet_velocity(xt, ys, fs, e1, e2, mu, 4.0)
    u_b = _ewald_stokeslet_velocity(xt, ys, fs, e1, e2, mu, 6.0, kmax=20)
    assert np.abs(u_a - u_b).max() < 1e-13
    M, m = 48, 24
    yp = periodic.proxy_points(c, 1.5, M)
    P = periodic.proxy_solution_operator(periodic.proxy_matrix(e1, e2, c, m, yp, mu))

    def oracle_velocity(shifts):
        g = periodic.near_discrepancy(e1, e2, c, m, ys, fs, mu)
        xi = periodic.apply_operator_exact(P, periodic.corrected_discrepancy(g, fs.sum(0), e1, e2, m))
        return periodic.near_velocity(xt, ys, fs, shifts, mu) + periodic.correction_velocity(xt, yp, xi, mu)

    scale = np.abs(u_a).max()
    d = oracle_velocity(periodic.image_shifts(e1, e2)) - u_a
    assert np.abs(d - d.mean(0)).max() < 1e-8 * scale
    plus = periodic.image_shifts(e1, e2, [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)])
    d = oracle_velocity(plus) - u_a
    assert np.abs(d - d.mean(0)).max() > 1e-4 * scale


@pytest.mark.parametrize("crossing", [False, True])
def test_contour_mu_eff_matches_stresslet(crossing):
    """Sec. 6.4 (Eq. contourdef, read with Gamma~ = {Gamma_1 - e1 - e2,
    Gamma_2 - e2, Gamma_3, Gamma_4 - e1}, the shifts that reproduce the
    per-node near sum): mu_eff from wall integrals half a cell or more from
    every source equals the particle-stress average (reading 9) to 1e-9, on a
    skewed cell with all bodies inside U and on one where a body crosses the
    bottom wall D, where the literal wall formula (Eq. mueff) no longer
    applies."""
    from oracle import bie as obie
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
                solver=dict(n_proxy=48, proxy_radius=1.5, n_coll=24))
    ou = obie.OperatorUtilde(oracle_suspension(cell), n_proxy=128, n_coll=32)
    st = np.linalg.solve(np.column_stack([e1, e2]), (ou.s.x - c).T).T
    assert (st[:, 1] < -0.5).any() == crossing
    sigma, _, res = obie.solve(ou, tol=1e-12)
    assert res <= 1e-12
    mu_s = ou.mu_eff(sigma)
    assert abs(ou.mu_eff_contour(sigma) - mu_s) < 1e-9
    wall = oracle_operator(cell, use_close=False).mu_eff_wall(sigma)
    if crossing:
        assert abs(wall - mu_s) > 1e-2
    else:
        assert abs(wall - mu_s) < 1e-8
