"""Pins of the oracle's star-shaped bodies (Sec. 8 Examples 4-5: boundaries
x(t) = r(t) (cos t, sin t) about the centre, here r(t) = r0 (1 + eps cos kt),
rotated by theta), against what the geometry fixes:

* the polar area (1/2) int r^2 dt = pi r0^2 (1 + eps^2 / 2), as the
  boundary integral (1/2) int (x - x^c) . n ds of the trapezoidal rule;
* the total curvature int kappa ds = 2 pi of a simple closed curve;
* first and second derivatives against central differences;
* the free-space jump identity K[n] = n / 2 and the force Gauss law on a star;
* Newton's closest point against dense sampling of the curve, and the fine
  rule of the close evaluation converged in its upsampling factor.
"""
import math

import numpy as np
import pytest

from oracle import close, geometry, kernels, periodic

STAR = dict(shape="star", r0=0.2, eps=0.5, k=4, xc=[0.3, -0.1], theta=0.3, n=512)


def test_star_area_and_total_curvature():
    g = geometry.body_nodes(STAR)
    area = 0.5 * ((g["x"] - np.asarray(STAR["xc"])) * g["n"]).sum(1) @ g["w"]
    r0, eps = STAR["r0"], STAR["eps"]
    assert abs(area - math.pi * r0 * r0 * (1 + eps * eps / 2)) < 1e-13
    assert abs(g["kappa"] @ g["w"] - 2 * math.pi) < 1e-11
    # a planted mistake: r'' of the wrong sign changes the total curvature
    b = dict(STAR)
    x, dx, ddx = geometry.curve_point(b, g["t"])
    sp = np.hypot(dx[:, 0], dx[:, 1])
    kappa_bad = (dx[:, 0] * (-ddx[:, 1]) - dx[:, 1] * (-ddx[:, 0])) / sp**3
    assert abs(kappa_bad @ g["w"] - 2 * math.pi) > 1.0


def test_star_derivatives_match_differences():
    t = np.linspace(0.1, 6.0, 13)
    h = 1e-5
    x, dx, ddx = geometry.curve_point(STAR, t)
    xp, _, _ = geometry.curve_point(STAR, t + h)
    xm, _, _ = geometry.curve_point(STAR, t - h)
    np.testing.assert_allclose(dx, (xp - xm) / (2 * h), atol=1e-8)
    np.testing.assert_allclose(ddx, (xp - 2 * x + xm) / h**2, atol=1e-4)


def test_star_jump_identity_and_gauss_law():
    g = geometry.body_nodes(STAR)
    x, nrm, w = g["x"], g["n"], g["w"]
    n = STAR["n"]

    def K(sig):
        q = sig * w[:, None]
        T = periodic.near_traction(x, nrm, x, q, [np.zeros(2)], self_index=np.arange(n))
        return T + kernels.traction_self(g["kappa"], g["tau"], q)
    np.testing.assert_allclose(K(nrm), 0.5 * nrm, atol=1e-10)
    sig = np.random.default_rng(0).normal(size=(n, 2))
    c = np.fft.fft(sig, axis=0)
    c[8:-7] = 0
    sig = np.real(np.fft.ifft(c, axis=0))
    np.testing.assert_allclose((K(sig) * w[:, None]).sum(0), -0.5 * (sig * w[:, None]).sum(0), atol=1e-10)


def test_star_closest_point_and_fine_rule():
    body = dict(STAR, n=128)
    g = geometry.body_nodes(body)
    # a target just outside the curve near a concave part, 2e-3 along the normal
    i = 37
    target = g["x"][i] + 2e-3 * g["n"][i] + 0.3 * (g["x"][i + 1] - g["x"][i])
    d, hl = close.closest_point(body, target, np.zeros(2), 2 * math.pi * i / body["n"])
    tt = np.linspace(0, 2 * math.pi, 200001)
    t0 = tt[np.hypot(*(geometry.curve_point(body, tt)[0] - target).T).argmin()]
    tt = np.linspace(t0 - 1e-3, t0 + 1e-3, 200001)  # sampling error ~(ds/2)^2 / (2 d) < 1e-14
    dense = np.hypot(*(geometry.curve_point(body, tt)[0] - target).T).min()
    assert abs(d - dense) < 1e-12 and 1e-3 < d < 3e-3
    sig = np.random.default_rng(1).normal(size=(body["n"], 2))
    f1 = close.fine_integral(body, sig, target, g["n"][i], np.zeros(2), close.fine_factor(hl, d))
    f2 = close.fine_integral(body, sig, target, g["n"][i], np.zeros(2), 2 * close.fine_factor(hl, d))
    assert np.abs(f1 - f2).max() < 1e-10 * np.abs(f2).max()
