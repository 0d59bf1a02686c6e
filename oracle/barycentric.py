"""Close evaluation by the paper's special quadrature (oracle, FP64; test
infrastructure: only tests/, the package's smoke() and bench.py's oracle legs
may import it), Sec. 6.3: barycentric-type ("globally compensated")
quadrature of Cauchy integrals, applied to the traction of the Stokes single
layer.

In complex notation (a vector v is v1 + i v2, r = z - zeta the target minus
the source point, n the target normal, sigma the density) the traction
kernel of Eq. (Gt) is

    G^t(z, zeta; n) sigma = -(1/(4 pi)) [ conj(n) conj(sigma) r / conj(r)^2
                                          + (conj(n) sigma + n conj(sigma)) / conj(r)
                                          + n sigma / r ],

so the integral over a closed curve Gamma of G^t sigma ds is made of three
integrals I1 = int sigma ds / (z - zeta), I2 = int conj(sigma) ds / (z - zeta)
and I3 = int sigma (conj(z) - conj(zeta)) ds / (z - zeta)^2:

    T(z) = -(1/(4 pi)) [ conj(n) conj(I3) + conj(n) conj(I2) + n conj(I1) + n I1 ].

With ds = dzeta / tau (tau the unit tangent), each is a Cauchy integral
C[h](z) = (1/(2 pi i)) oint h(zeta) / (zeta - z) dzeta or its derivative
C'[h](z) = (1/(2 pi i)) oint h / (zeta - z)^2 dzeta, with h = g / tau:

    I1 = -2 pi i C[sigma / tau],   I2 = -2 pi i C[conj(sigma) / tau],
    I3 = 2 pi i (conj(z) C'[sigma / tau] - C'[sigma conj(zeta) / tau]).

For z outside Gamma, C[h] is analytic in the exterior and vanishes at
infinity.  Its boundary values from the exterior follow from the Plemelj
formula, phi(zeta0) = (1/(2 pi i)) oint (h(zeta) - h(zeta0)) / (zeta - zeta0)
dzeta, whose integrand is smooth, so the trapezoidal rule on the N nodes is
spectrally accurate (the k = j term is its limit h'(t_j) 2 pi / N).  A
function v analytic outside Gamma with v(inf) = 0 satisfies
oint v / (zeta - z) dzeta = -2 pi i v(z) while oint dzeta / (zeta - z) = 0;
subtracting v(z) times the second from the first before discretising gives
the compensated (barycentric) exterior rule

    v(z) = sum_j v_j W_j / (sum_j W_j - 2 pi i),   W_j = w_j / (zeta_j - z),

w_j = zeta'(t_j) 2 pi / N, whose numerator and denominator carry the same
near-singular quadrature error, so it stays accurate as z approaches Gamma.
C[h] takes it with v_j = phi_j, and C'[h] with v_j = phi'_j, the tangential
derivative dphi/dt / zeta'(t) (by FFT).  The result is the integral of G^t
times the trigonometric interpolant of the nodal density over the exact
curve, the quantity the close-evaluation blocks of the solver are defined to
be (oracle/close.py evaluates the same quantity by brute force).
"""
import numpy as np

from . import geometry, kernels


def curve(body, shift=(0.0, 0.0)):
    """Nodes zeta_j, derivative zeta'(t_j) and unit tangent of a body's
    boundary (translated by shift), complex, at t_j = 2 pi j / N."""
    n = body["n"]
    t = 2.0 * np.pi * np.arange(n) / n
    x, dx, _ = geometry.curve_point(body, t)
    zeta = (x[:, 0] + shift[0]) + 1j * (x[:, 1] + shift[1])
    dz = dx[:, 0] + 1j * dx[:, 1]
    return zeta, dz, dz / np.abs(dz)


def spectral_dt(v):
    """d/dt of the trigonometric interpolant of samples v (n, ...) at
    t_k = 2 pi k / n, at the same points (the Nyquist mode, for even n,
    contributes nothing)."""
    v = np.asarray(v)
    n = v.shape[0]
    k = np.fft.fftfreq(n, d=1.0 / n)
    if n % 2 == 0:
        k[n // 2] = 0.0
    shape = (n,) + (1,) * (v.ndim - 1)
    return np.fft.ifft(1j * k.reshape(shape) * np.fft.fft(v, axis=0), axis=0)


def exterior_values(zeta, dz, h):
    """Boundary values from the exterior of C[h] at the nodes (columns of h
    are separate functions): (1/(2 pi i)) [ sum_{k != j} (h_k - h_j) w_k /
    (zeta_k - zeta_j) + h'(t_j) 2 pi / N ], w_k = zeta'(t_k) 2 pi / N."""
    h = np.asarray(h, dtype=np.complex128)
    one = h.ndim == 1
    if one:
        h = h[:, None]
    n = zeta.shape[0]
    w = dz * (2.0 * np.pi / n)
    diff = zeta[None, :] - zeta[:, None]        # [j, k] = zeta_k - zeta_j
    np.fill_diagonal(diff, 1.0)
    inv = w[None, :] / diff
    np.fill_diagonal(inv, 0.0)
    phi = np.empty_like(h)
    dh = spectral_dt(h)
    for c in range(h.shape[1]):
        hc = h[:, c]
        phi[:, c] = (inv @ hc - inv.sum(1) * hc + dh[:, c] * (2.0 * np.pi / n)) / (2j * np.pi)
    return phi[:, 0] if one else phi


def exterior_barycentric(zeta, dz, v, z):
    """v(z) for z outside the curve, from the boundary values v_j of a
    function analytic outside it that vanishes at infinity (columns of v are
    separate functions)."""
    n = zeta.shape[0]
    W = dz * (2.0 * np.pi / n) / (zeta - z)
    return (W @ v) / (W.sum() - 2j * np.pi)


def slp_traction(body, sigma_b, x, nx, shift=(0.0, 0.0)):
    """int over the exact curve of `body` (translated by shift) of
    G^t(x, y; nx) sigma^(y) ds_y, sigma^ the trigonometric interpolant of the
    nodal density sigma_b (n_b, 2), for a target x outside the curve, by the
    compensated barycentric rule."""
    zeta, dz, tau = curve(body, shift)
    s = sigma_b[:, 0] + 1j * sigma_b[:, 1]
    h = np.stack([s / tau, np.conj(s) / tau, s * np.conj(zeta) / tau], axis=1)
    phi = exterior_values(zeta, dz, h)
    dphi = spectral_dt(phi) / dz[:, None]
    z = x[0] + 1j * x[1]
    C = exterior_barycentric(zeta, dz, phi, z)       # C[h] for the three h
    Cp = exterior_barycentric(zeta, dz, dphi, z)     # C'[h]
    I1 = -2j * np.pi * C[0]
    I2 = -2j * np.pi * C[1]
    I3 = 2j * np.pi * (np.conj(z) * Cp[0] - Cp[2])
    n = nx[0] + 1j * nx[1]
    T = -(np.conj(n) * np.conj(I3) + np.conj(n) * np.conj(I2) + n * np.conj(I1) + n * I1) / (4.0 * np.pi)
    return np.array([T.real, T.imag])


def correction(body, sigma_b, x, nx, shift=(0.0, 0.0)):
    """The close-evaluation correction for target x and one body image: the
    barycentric integral minus the body's smooth N_b-point rule."""
    nodes = geometry.body_nodes(body)
    r = np.asarray(x)[None, :] - (nodes["x"] + np.asarray(shift)[None, :])
    smooth = kernels.traction(r, np.asarray(nx)[None, :], sigma_b * nodes["w"][:, None]).sum(0)
    return slp_traction(body, sigma_b, np.asarray(x, dtype=np.float64), np.asarray(nx, dtype=np.float64),
                        shift) - smooth
