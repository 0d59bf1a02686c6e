"""Pins of the oracle's BIE operator, solver and post-processing against what
the paper and the physics fix (Sec. 3-7):

* free-space jump relation + uniqueness: K[n] = n/2 on any closed curve, and
  the Gauss laws int K sigma = -1/2 int sigma (force) and its torque analogue;
* the solved density carries zero net force and torque per body (Lemma after
  Eq. BIEPerturbed2) and the flow inside every body is exactly the extracted
  rigid motion (Eq. RigidBodyMotion);
* dilute limits: a circle rotates at -gamma/2, an ellipse at Jeffery's rate,
  and mu_eff = mu (1 + 2 phi) (2D Einstein law) for dilute circles;
* the stresslet mu_eff equals the wall formula Eq. (mueff) when D is clear;
* spectral convergence in N; GMRES matches a dense direct solve;
* time stepping: the lattice of Sec. 7 and first order in dt.
"""
import math

import numpy as np
import pytest

from oracle import bie, geometry, kernels, periodic
from paper_1912_04501_gb300 import workloads
from tests.conftest import oracle_operator, oracle_suspension


def one_body(a, b, theta=0.0, n=64, xc=(0.5, 0.5), e2=(0.0, 1.0), M=48, m=24):
    cell = dict(e1=[1.0, 0.0], e2=list(e2), centre=[0.5, 0.5], mu=1.0, gamma=1.0,
                bodies=[dict(a=a, b=b, xc=list(xc), theta=theta, n=n)],
                solver=dict(n_proxy=M, proxy_radius=1.5, n_coll=m))
    return oracle_operator(cell)


@pytest.mark.parametrize("shape", [(0.3, 0.1, 0.4, 64), (0.2, 0.2, 0.0, 32), (0.1, 0.25, 2.0, 96)])
def test_free_space_jump_identities(shape):
    a, b, th, n = shape
    g = geometry.ellipse_nodes(a, b, [0.1, -0.2], th, n)
    x, nrm, w = g["x"], g["n"], g["w"]
    def K(sig):
        q = sig * w[:, None]
        T = periodic.near_traction(x, nrm, x, q, [np.zeros(2)], self_index=np.arange(n))
        return T + kernels.traction_self(g["kappa"], g["tau"], q)
    np.testing.assert_allclose(K(nrm), 0.5 * nrm, atol=1e-13)
    sig = np.random.default_rng(0).normal(size=(n, 2))
    # band-limit the random density so the trapezoidal rule is exact enough
    from oracle.close import trig_interp
    c = np.fft.fft(sig, axis=0)
    c[6:-5] = 0
    sig = np.real(np.fft.ifft(c, axis=0))
    Ks = K(sig)
    np.testing.assert_allclose((Ks * w[:, None]).sum(0), -0.5 * (sig * w[:, None]).sum(0), atol=1e-12)
    xc = np.array([0.1, -0.2])
    perp = lambda v: np.stack([-v[:, 1], v[:, 0]], 1)
    tq = lambda f: (perp(x - xc) * f * w[:, None]).sum()
    assert abs(tq(Ks) + 0.5 * tq(sig)) < 1e-12


def test_gmres_matches_dense_solve():
    cell = workloads.small_cell(n_bodies=2, nodes=40, seed=1)
    op = oracle_operator(cell)
    n2 = 2 * op.s.N
    A = np.stack([op.matvec(e) for e in np.eye(n2)], axis=1)
    b = op.rhs().ravel()
    x_dense = np.linalg.solve(A, b)
    x, it, res = bie.solve(op, tol=1e-12)
    assert res < 1e-12
    np.testing.assert_allclose(x.ravel(), x_dense, atol=1e-11 * np.abs(x_dense).max())
    assert np.linalg.cond(A) < 1e3


def test_solution_invariants_and_rigid_interior():
    cell = workloads.small_cell(n_bodies=3, nodes=64, seed=2, e2=(0.25, 1.0))
    op = oracle_operator(cell, n_proxy=48, n_coll=24)
    s = op.s
    sigma, it, res = bie.solve(op)
    assert res <= 1e-10
    _, F, tau = op.density_moments(sigma)
    assert np.abs(F).max() < 1e-10 and np.abs(tau).max() < 1e-10
    v, om = op.body_velocities(sigma)
    q, _, _ = op.density_moments(sigma)
    xi, _ = op.proxy_strengths(q)
    for b, bd in enumerate(s.bodies):
        # interior points at half the semi-axes
        t = np.linspace(0, 2 * np.pi, 7, endpoint=False)
        c, sn = math.cos(bd["theta"]), math.sin(bd["theta"])
        px, py = 0.5 * bd["a"] * np.cos(t), 0.5 * bd["b"] * np.sin(t)
        pts = np.stack([bd["xc"][0] + c * px - sn * py, bd["xc"][1] + sn * px + c * py], 1)
        u = periodic.near_velocity(pts, s.x, q, op.shifts, s.mu)
        u += periodic.correction_velocity(pts, op.yp, xi, s.mu)
        u -= periodic.correction_velocity(s.centre[None], op.yp, xi, s.mu)
        u[:, 0] += s.gamma * pts[:, 1]
        rigid = v[b] + om[b] * np.stack([-(pts[:, 1] - bd["xc"][1]), pts[:, 0] - bd["xc"][0]], 1)
        np.testing.assert_allclose(u, rigid, atol=1e-9)


def test_dilute_circle_rotates_at_half_shear():
    for r in (0.05, 0.02):
        op = one_body(r, r, n=32, M=16, m=16)
        sigma, _, _ = bie.solve(op)
        v, om = op.body_velocities(sigma)
        phi = math.pi * r * r
        assert abs(om[0] + 0.5) < 5 * phi
        np.testing.assert_allclose(v[0], [0.5, 0.0], atol=1e-12)


def test_jeffery_rate_dilute_ellipse():
    a0, b0, th = 0.2, 0.1, 0.4
    jeff = -(a0**2 * math.sin(th) ** 2 + b0**2 * math.cos(th) ** 2) / (a0**2 + b0**2)
    errs = []
    for eps in (0.4, 0.2, 0.1):
        op = one_body(a0 * eps, b0 * eps, th, n=64, M=16, m=16)
        sigma, _, _ = bie.solve(op)
        errs.append(abs(op.body_velocities(sigma)[1][0] - jeff))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3


def test_einstein_viscosity():
    slopes = []
    for r in (0.04, 0.02):
        op = one_body(r, r, n=32, M=16, m=16)
        sigma, _, _ = bie.solve(op)
        phi = math.pi * r * r
        slopes.append((op.mu_eff(sigma) - 1.0) / phi)
    assert abs(slopes[1] - 2.0) < 0.01
    assert abs(slopes[1] - 2.0) < abs(slopes[0] - 2.0)


def test_mu_eff_stresslet_equals_wall_formula():
    cell = workloads.config1()
    cell["bodies"][0]["theta"] = 0.7
    op = oracle_operator(cell, n_proxy=48, n_coll=24)
    sigma, _, _ = bie.solve(op)
    assert abs(op.mu_eff(sigma) - op.mu_eff_wall(sigma, 128)) < 1e-8


def test_spectral_convergence_in_n():
    om = []
    for n in (24, 48, 96):
        op = one_body(0.2, 0.1, 0.3, n=n, M=16, m=16)
        sigma, _, _ = bie.solve(op)
        om.append(op.body_velocities(sigma)[1][0])
    d1, d2 = abs(om[0] - om[2]), abs(om[1] - om[2])
    assert d2 < 1e-3 * d1 and d2 < 1e-10


def test_lattice_rounding_and_wrap():
    e1, e2 = geometry.lattice_at([1.0, 0.0], [0.0, 1.0], 1.0, 0.3)
    np.testing.assert_allclose(e2, [0.3, 1.0])
    e1, e2 = geometry.lattice_at([1.0, 0.0], [0.0, 1.0], 1.0, 0.7)
    np.testing.assert_allclose(e2, [-0.3, 1.0], atol=1e-15)
    e1, e2 = geometry.lattice_at([1.0, 0.0], [0.0, 1.0], 2.0, 0.75)  # gamma t = 1.5 rounds to 2
    np.testing.assert_allclose(e2, [-0.5, 1.0])
    p = geometry.wrap_into_cell([1.2, -0.1], np.array([1.0, 0.0]), np.array([0.3, 1.0]), np.array([0.5, 0.5]))
    ab = np.linalg.solve(np.array([[1.0, 0.3], [0.0, 1.0]]), p - 0.5)
    assert np.all(ab >= -0.5) and np.all(ab < 0.5)


def test_euler_first_order():
    cell = dict(e1=[1.0, 0.0], e2=[0.0, 1.0], centre=[0.5, 0.5], mu=1.0, gamma=1.0,
                bodies=[dict(a=0.2, b=0.1, xc=[0.45, 0.55], theta=0.2, n=48),
                        dict(a=0.12, b=0.08, xc=[0.05, 0.1], theta=1.0, n=40)])
    kw = dict(n_proxy=16, proxy_radius=1.5, n_coll=16)
    T = 0.04
    finals = []
    for dt in (0.02, 0.01, 0.005):
        s = oracle_suspension(cell)
        t = 0.0
        for _ in range(int(round(T / dt))):
            s, t, out = bie.euler_step(s, cell["e2"], t, dt, kw)
        finals.append(np.array([b["theta"] for b in s.bodies]))
    e1, e2 = np.abs(finals[0] - finals[2]).max(), np.abs(finals[1] - finals[2]).max()
    assert 2.2 < e1 / e2 < 3.8  # (2 dt - dt/2) / (dt - dt/2) = 3 for first order


def _circle_cell(r, xc, e2=(0.0, 1.0)):
    return dict(e1=[1.0, 0.0], e2=list(e2), centre=[0.5, 0.5], mu=1.0, gamma=1.0,
                bodies=[dict(a=r, b=r, xc=list(xc), theta=0.0, n=32)])


EULER_KW = dict(n_proxy=16, proxy_radius=1.5, n_coll=16)


def test_euler_step_dilute_circle_closed_form():
    """Sec. 7, forward Euler: one step of a dilute circle moves its centre by
    dt u0(x^c) = dt (gamma y_c, 0) and turns it by -dt gamma / 2 (the dilute
    rotation rate), up to O(phi) corrections.  A flipped sign of either update
    (or of the background flow) misses by 2 dt |v| or dt gamma."""
    r, dt = 0.01, 0.05
    phi = math.pi * r * r
    cell = _circle_cell(r, (0.5, 0.7))
    s = oracle_suspension(cell)
    s1, t1, out = bie.euler_step(s, cell["e2"], 0.0, dt, EULER_KW)
    assert t1 == dt
    dx = np.asarray(s1.bodies[0]["xc"]) - np.array([0.5, 0.7])
    np.testing.assert_allclose(dx, [dt * 0.7, 0.0], atol=10 * phi * dt)
    assert abs((s1.bodies[0]["theta"] - 0.0) - (-0.5 * dt)) < 10 * phi * dt
    # the lattice of the new state is the one at t + dt (Sec. 7: the top of the
    # cell moves with u0, e2 = (gamma t L2, L2)), not the one at t
    np.testing.assert_allclose(s1.e2, [dt, 1.0], atol=1e-15)
    np.testing.assert_allclose(s1.e1, [1.0, 0.0], atol=0)


def test_euler_steps_lattice_and_wrap():
    """After n steps the lattice is e2(n dt) with round() reducing the skew
    (Sec. 7), and a centre that leaves the cell re-enters through the opposite
    wall: a dilute circle at y_c = 0.9 moving right with speed ~0.9."""
    r, dt = 0.01, 0.2
    cell = _circle_cell(r, (0.8, 0.9))
    s = oracle_suspension(cell)
    t = 0.0
    xs = []
    for _ in range(3):
        s, t, out = bie.euler_step(s, cell["e2"], t, dt, EULER_KW)
        xs.append((np.asarray(s.bodies[0]["xc"]), s.e2.copy()))
    # gamma t = 0.6 rounds to 1: e2 = (0.6 - 1, 1)
    np.testing.assert_allclose(s.e2, [-0.4, 1.0], atol=1e-14)
    np.testing.assert_allclose(t, 0.6, atol=1e-15)
    # unwrapped, the centre would be at 0.8 + 3 * 0.2 * 0.9 = 1.34; it is the
    # same point shifted by -e1 = (-1, 0) of the lattice it was wrapped in
    phi = math.pi * r * r
    np.testing.assert_allclose(xs[-1][0], [0.34, 0.9], atol=30 * phi * dt)
    for x, e2 in xs:
        ab = np.linalg.solve(np.column_stack([[1.0, 0.0], e2]), x - 0.5)
        assert np.all(ab >= -0.5) and np.all(ab < 0.5)


def test_euler_uses_velocities_of_the_current_state():
    """Forward Euler (Sec. 7) advances with F(t, s(t)): the step equals dt times
    the rigid motion extracted from an independent solve on the geometry at t
    (not at t + dt), for two interacting ellipses in a skewed cell."""
    cell = dict(e1=[1.0, 0.0], e2=[0.2, 1.0], centre=[0.5, 0.5], mu=1.0, gamma=1.0,
                bodies=[dict(a=0.2, b=0.1, xc=[0.45, 0.55], theta=0.2, n=48),
                        dict(a=0.12, b=0.08, xc=[0.05, 0.1], theta=1.0, n=40)])
    dt = 0.01
    s0 = oracle_suspension(cell)
    op = oracle_operator(dict(cell, solver=dict(n_proxy=16, proxy_radius=1.5, n_coll=16)))
    sigma, _, _ = bie.solve(op)
    v, om = op.body_velocities(sigma)
    s1, t1, out = bie.euler_step(s0, cell["e2"], 0.0, dt, EULER_KW)
    for b in range(2):
        new = np.asarray(s1.bodies[b]["xc"])
        moved = np.asarray(cell["bodies"][b]["xc"]) + dt * v[b]
        d = new - moved  # equal up to a lattice vector of the new cell
        ab = np.linalg.solve(np.column_stack([s1.e1, s1.e2]), d)
        np.testing.assert_allclose(ab, np.round(ab), atol=1e-12)
        assert abs(s1.bodies[b]["theta"] - (cell["bodies"][b]["theta"] + dt * om[b])) < 1e-12
    # the velocities differ measurably between t and t + dt, so a step that
    # used the new geometry's velocities would fail the check above
    op1 = oracle_operator(dict(cell, e2=list(s1.e2), bodies=s1.bodies,
                               solver=dict(n_proxy=16, proxy_radius=1.5, n_coll=16)))
    v1, om1 = op1.body_velocities(bie.solve(op1)[0])
    assert np.abs(om1 - om).max() * dt > 1e-9
