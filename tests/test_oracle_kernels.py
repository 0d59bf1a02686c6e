"""Pins of the oracle's free-space kernels (Sec. 4.1) against the mathematics:
the traction kernel must be the stress of the Stokeslet (Eqs. Gv, Gp, Gt with
the stress of Sec. 3), satisfy Gauss' law, and the Stokeslet must solve the
Stokes equations.  A dropped factor, a wrong sign or a transposed index in any
of the three kernels fails one of these."""
import numpy as np
import pytest

from oracle import kernels

MU = 0.7


def _fd_grad(fun, x, h=1e-5):
    """Central differences: d fun_i / d x_k -> (..., i, k)."""
    g = []
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        g.append((fun(x + e) - fun(x - e)) / (2 * h))
    return np.stack(g, axis=-1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_traction_is_stokeslet_stress(seed):
    rng = np.random.default_rng(seed)
    y = rng.normal(size=2)
    f = rng.normal(size=2)
    x = y + rng.normal(size=2) * 0.7
    nx = rng.normal(size=2)
    nx /= np.linalg.norm(nx)
    u = lambda z: kernels.stokeslet(z - y, f, MU)
    p = kernels.stokeslet_pressure(x - y, f)
    du = _fd_grad(u, x)  # du[i, k] = d u_i / d x_k
    sigma = -p * np.eye(2) + MU * (du + du.T)
    want = sigma @ nx
    got = kernels.traction(x - y, nx, f)
    np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-9)


def test_traction_gauss_law():
    """Force balance on a disc around a point force: the outward traction
    integrates to -f (Lemma on net quantities, Sec. 4.1)."""
    f = np.array([0.3, -0.6])
    y = np.array([0.2, 0.1])
    k = 400
    th = 2 * np.pi * np.arange(k) / k
    for R in (0.05, 1.0, 7.0):
        x = y + R * np.stack([np.cos(th), np.sin(th)], 1)
        n = (x - y) / R
        t = kernels.traction(x - y, n, f[None, :])
        np.testing.assert_allclose(t.sum(0) * (2 * np.pi * R / k), -f, atol=1e-13)


def test_stokeslet_solves_stokes():
    rng = np.random.default_rng(5)
    y = np.zeros(2)
    f = rng.normal(size=2)
    h = 1e-3
    for _ in range(5):
        x = rng.normal(size=2)
        u = lambda z: kernels.stokeslet(z - y, f, MU)
        p = lambda z: kernels.stokeslet_pressure(z - y, f)
        lap = sum((u(x + h * e) - 2 * u(x) + u(x - h * e)) / h**2 for e in np.eye(2))
        gp = np.array([(p(x + h * e) - p(x - h * e)) / (2 * h) for e in np.eye(2)])
        np.testing.assert_allclose(-MU * lap + gp, 0, atol=1e-5)
        hd = 1e-5
        div = sum((u(x + hd * e)[k] - u(x - hd * e)[k]) / (2 * hd) for k, e in enumerate(np.eye(2)))
        assert abs(div) < 1e-8


def test_stokeslet_vorticity():
    rng = np.random.default_rng(7)
    for _ in range(4):
        y, f, x = rng.normal(size=2), rng.normal(size=2), rng.normal(size=2)
        du = _fd_grad(lambda z: kernels.stokeslet(z - y, f, MU), x)
        np.testing.assert_allclose(kernels.stokeslet_vorticity(x - y, f, MU), du[1, 0] - du[0, 1],
                                   rtol=1e-7)


def test_point_force_far_field_log():
    """G is 1/(4 pi mu) (-log r I + r r^T / r^2): at r = 1 along e_x the xx
    entry is 1/(4 pi mu), the yy entry 0."""
    g = kernels.stokeslet(np.array([[1.0, 0.0], [1.0, 0.0]]), np.eye(2), MU)
    np.testing.assert_allclose(g, np.diag([1 / (4 * np.pi * MU), 0.0]), atol=1e-15)
