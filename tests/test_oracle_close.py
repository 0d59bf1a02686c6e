"""Pins of the oracle's close-evaluation correction (Sec. 6.3).

* The trigonometric interpolant reproduces trigonometric polynomials.
* A single layer with density n has zero traction everywhere outside the
  curve and traction nu (pressure -1) inside (jump relation + uniqueness): the
  corrected integral reproduces both at distances far below the node spacing,
  where the smooth rule is O(1) wrong.
* Against an independent adaptive quadrature (scipy quad) of the exact
  integrand at a close target.
* The correction is negligible beyond the 10h zone.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import close, geometry, kernels


def test_trig_interp_exact():
    n = 16
    t = 2 * np.pi * np.arange(n) / n
    f = lambda s: 0.3 + np.cos(3 * s) - 0.7 * np.sin(7 * s) + 0.25 * np.cos(8 * s)
    nf = 64
    tf = 2 * np.pi * np.arange(nf) / nf
    np.testing.assert_allclose(close.trig_interp(f(t), nf), f(tf), atol=1e-14)


BODY = dict(a=0.2, b=0.1, xc=[0.0, 0.0], theta=0.3, n=64)


def _targets(d, inside):
    """Points at distance ~d from the ellipse, just outside (or inside)."""
    g = geometry.ellipse_nodes(BODY["a"], BODY["b"], BODY["xc"], BODY["theta"], 997)
    k = np.arange(5, 997, 83)
    sgn = -1.0 if inside else 1.0
    return g["x"][k] + sgn * d * g["n"][k]


@pytest.mark.parametrize("d", [1e-2, 1e-3, 1e-4])
def test_single_layer_of_normal(d):
    # the unit normal is not a trigonometric polynomial; 128 nodes resolve it
    # to rounding, so what remains is the close-evaluation error alone
    body = dict(BODY, n=128)
    g = geometry.ellipse_nodes(body["a"], body["b"], body["xc"], body["theta"], body["n"])
    h = g["w"].sum() / body["n"]
    rng = np.random.default_rng(0)
    for inside in (False, True):
        for x in _targets(d, inside):
            nu = rng.normal(size=2)
            nu /= np.linalg.norm(nu)
            T = close.fine_integral(body, g["n"], x, nu, np.zeros(2), close.fine_factor(h, d))
            want = nu if inside else np.zeros(2)
            np.testing.assert_allclose(T, want, atol=1e-11)
            if d < h / 5:
                smooth = kernels.traction(x[None] - g["x"], nu[None], g["n"] * g["w"][:, None]).sum(0)
                assert np.abs(smooth - want).max() > 1e-3


def test_against_adaptive_quadrature():
    g = geometry.ellipse_nodes(BODY["a"], BODY["b"], BODY["xc"], BODY["theta"], BODY["n"])
    n = BODY["n"]
    t = g["t"]
    sig = np.stack([np.cos(t) + 0.3 * np.sin(5 * t), 0.5 - np.sin(2 * t) + 0.1 * np.cos(9 * t)], 1)
    x = _targets(3e-4, False)[2]
    nu = np.array([0.6, 0.8])
    h = g["w"].sum() / n
    got = close.fine_integral(BODY, sig, x, nu, np.zeros(2), close.fine_factor(h, 3e-4))

    def integrand(s, comp):
        y, sp = geometry.ellipse_point(BODY["a"], BODY["b"], BODY["xc"], BODY["theta"], [s])
        f = np.array([np.cos(s) + 0.3 * np.sin(5 * s), 0.5 - np.sin(2 * s) + 0.1 * np.cos(9 * s)])
        return kernels.traction(x - y[0], nu, f)[comp] * sp[0]
    want = [integrate.quad(integrand, 0, 2 * np.pi, args=(c,), limit=2000, epsabs=1e-14, epsrel=1e-13,
                           points=np.linspace(0, 2 * np.pi, 65)[1:-1])[0] for c in range(2)]
    np.testing.assert_allclose(got, want, atol=1e-10, rtol=1e-10)


def test_correction_vanishes_far_away():
    g = geometry.ellipse_nodes(BODY["a"], BODY["b"], BODY["xc"], BODY["theta"], BODY["n"])
    h = g["w"].sum() / BODY["n"]
    sig = np.random.default_rng(2).normal(size=(BODY["n"], 2))
    c = np.fft.fft(sig, axis=0)
    c[10:-9] = 0
    sig = np.real(np.fft.ifft(c, axis=0))
    for x in _targets(10 * h, False):
        nu = np.array([1.0, 0.0])
        fine = close.fine_integral(BODY, sig, x, nu, np.zeros(2), 8)
        coarse = kernels.traction(x[None] - g["x"], nu[None], sig * g["w"][:, None]).sum(0)
        assert np.abs(fine - coarse).max() < 1e-12


def test_fine_rule_converged_at_chosen_factor():
    """For every close pair of the two-ellipse cell at gap 2e-3 the oracle's
    fine rule agrees with the rule of twice the resolution."""
    from paper_1912_04501_gb300 import workloads
    from tests.conftest import oracle_operator
    cell = workloads.two_ellipses(2e-3, 192)
    op = oracle_operator(cell)
    s = op.s
    sig = np.random.default_rng(3).normal(size=(s.N, 2))
    assert len(op.close.pairs) > 10
    for (i, b, sh, d, hl) in op.close.pairs:
        bd = s.bodies[b]
        sl = slice(s.offsets[b], s.offsets[b + 1])
        rho = close.fine_factor(hl, d)
        a = close.fine_integral(bd, sig[sl], s.x[i], s.n[i], sh, rho)
        c = close.fine_integral(bd, sig[sl], s.x[i], s.n[i], sh, 2 * rho)
        assert np.abs(a - c).max() < 1e-13


def test_closest_point_matches_dense_sampling():
    from oracle import close as cl
    body = dict(a=0.3, b=0.1, xc=[0.2, -0.1], theta=0.7, n=64)
    rng = np.random.default_rng(5)
    t = np.linspace(0, 2 * np.pi, 400001)
    for _ in range(10):
        k = rng.integers(64)
        g = geometry.ellipse_nodes(body["a"], body["b"], body["xc"], body["theta"], 64)
        x = g["x"][k] + rng.uniform(1e-4, 2e-2) * g["n"][k] + rng.normal(size=2) * 1e-3
        d, hl = cl.closest_point(body, x, np.zeros(2), 2 * np.pi * k / 64)
        y, sp = geometry.ellipse_point(body["a"], body["b"], body["xc"], body["theta"], t)
        dd = np.sqrt(((y - x) ** 2).sum(1))
        # the sampled minimum overestimates by up to (ds)^2 / (8 d) ~ 2e-9
        assert -1e-8 < dd.min() - d < 1e-8
        assert abs(hl - 2 * np.pi * sp[dd.argmin()] / 64) < 1e-6
