"""Free-space Stokes kernels in 2D (oracle, FP64), Sec. 4.1.

Eq. (Gv):  G_ij(x, y) = (1/(4 pi mu)) (delta_ij log(1/r) + r_i r_j / r^2)
Eq. (Gp):  G^p_j(x, y) = (1/(2 pi)) r_j / r^2
Eq. (Gt):  G^t_ik(x, y) = -(1/pi) r_i r_k (r . n_x) / r^4
with r = x - y, r = |r|, and n_x the unit normal at the TARGET x.

All functions take arrays of displacement vectors r (..., 2) and return the
kernel applied to a strength vector f (..., 2).
"""
import numpy as np


def _dot(a, b):
    return a[..., 0] * b[..., 0] + a[..., 1] * b[..., 1]


def stokeslet(r, f, mu):
    """Velocity G(x, y) f of a point force f at y, Eq. (Gv)."""
    r2 = _dot(r, r)
    rf = _dot(r, f)
    return (-0.5 * np.log(r2)[..., None] * f + r * (rf / r2)[..., None]) / (4.0 * np.pi * mu)


def stokeslet_pressure(r, f):
    """Pressure G^p(x, y) . f, Eq. (Gp)."""
    return _dot(r, f) / _dot(r, r) / (2.0 * np.pi)


def traction(r, nx, f):
    """Traction G^t(x, y) f on a surface through x with normal nx, Eq. (Gt)."""
    r2 = _dot(r, r)
    c = _dot(r, nx) * _dot(r, f) / (r2 * r2)
    return (-1.0 / np.pi) * r * c[..., None]


def stokeslet_vorticity(r, f, mu):
    """curl u = d u2/dx1 - d u1/dx2 of u = G(x, y) f.

    Differentiating Eq. (Gv) term by term, the r_i r_j / r^2 part contributes
    equal cross derivatives that cancel in the curl, leaving the log part:
    curl u = (r2 f1 - r1 f2) / (2 pi mu r^2).
    """
    r2 = _dot(r, r)
    return (r[..., 1] * f[..., 0] - r[..., 0] * f[..., 1]) / (2.0 * np.pi * mu * r2)


def traction_self(kappa, tau, f):
    """Smooth on-curve limit of Eq. (Gt) as y -> x along the curve.

    With r ~ -x' dt and (r . n) ~ -(x'' . n) dt^2 / 2 the ratio
    r_i r_k / r^2 -> tau_i tau_k and (r . n)/r^2 -> kappa/2, so
    G^t(x, x) f = -(kappa / (2 pi)) tau (tau . f).
    """
    return -(kappa / (2.0 * np.pi))[..., None] * tau * _dot(tau, f)[..., None]
