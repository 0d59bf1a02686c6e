"""Close-evaluation correction (oracle, FP64), Sec. 6.3 and its remark on the
two-phase solver.

For a target x within close_factor * h_b of source body b (h_b = perimeter /
N_b), the smooth N_b-point rule for int_{Gamma_b} G^t(x, y; n_x) sigma(y) ds_y
loses accuracy.  The paper replaces it by a special quadrature that is exact
for the interpolant of the nodal density.  The oracle computes the quantity
such a rule converges to by its definition: the integral, over the exact
curve, of G^t times the trigonometric interpolant sigma^ of the nodal values,
evaluated by the trapezoidal rule on a grid fine enough (local fine spacing
<= d / 8, d the distance to the curve, and at least 4x the nodes) that its own
error is below double-precision rounding.
The correction added to the near sum is that integral minus the smooth
N_b-point rule's contribution from the same body image.
"""
import math

import numpy as np

from . import geometry, kernels


def trig_interp(v, nf):
    """Values at t_f = 2 pi f / nf of the trigonometric interpolant of the
    samples v (n, ...) at t_k = 2 pi k / n.  For even n the Nyquist
    coefficient is split equally between the +n/2 and -n/2 modes."""
    v = np.asarray(v, dtype=np.float64)
    n = v.shape[0]
    c = np.fft.fft(v, axis=0) / n
    big = np.zeros((nf,) + v.shape[1:], dtype=np.complex128)
    h = n // 2
    if n % 2 == 0:
        big[:h] = c[:h]
        big[nf - h + 1:] = c[h + 1:]
        big[h] = 0.5 * c[h]
        big[nf - h] = 0.5 * c[h]
    else:
        big[:h + 1] = c[:h + 1]
        big[nf - h:] = c[h + 1:]
    return np.real(np.fft.ifft(big, axis=0) * nf)


def fine_factor(h, d):
    """Upsampling factor of the oracle's fine rule: a power of two >= 4 with
    h / factor <= d / 8 (h the local node spacing, d the distance to the
    curve)."""
    need = 8.0 * h / max(d, 1e-300)
    return max(4, 1 << max(0, math.ceil(math.log2(need))))


def closest_point(body, x, shift, t0, n_iter=8):
    """Distance from x to the exact curve of `body` translated by shift, and
    the local node spacing 2 pi |x'(t*)| / N_b there, by Newton's method on
    the stationarity condition (y(t) - x) . y'(t) = 0 started at t0 (the
    parameter of the nearest node); steps are capped at one node spacing."""
    if body.get("shape", "ellipse") == "star":
        dt_max = 2.0 * math.pi / body["n"]
        t = t0
        xs = np.asarray(x, dtype=np.float64) - np.asarray(shift, dtype=np.float64)
        for _ in range(n_iter):
            y, dy, ddy = geometry.curve_point(body, [t])
            d = y[0] - xs
            g = d @ dy[0]
            gp = dy[0] @ dy[0] + d @ ddy[0]
            step = g / gp if gp > 0 else math.copysign(dt_max, g)
            t -= max(-dt_max, min(dt_max, step))
        y, dy, _ = geometry.curve_point(body, [t])
        return float(np.hypot(*(y[0] - xs))), 2.0 * math.pi * float(np.hypot(*dy[0])) / body["n"]
    a, b, th = body["a"], body["b"], body["theta"]
    c, s = math.cos(th), math.sin(th)
    px = x[0] - body["xc"][0] - shift[0]
    py = x[1] - body["xc"][1] - shift[1]
    u, v = c * px + s * py, -s * px + c * py   # target in the body frame
    dt_max = 2.0 * math.pi / body["n"]
    t = t0
    for _ in range(n_iter):
        g = (b * b - a * a) * math.sin(t) * math.cos(t) + a * u * math.sin(t) - b * v * math.cos(t)
        gp = (b * b - a * a) * math.cos(2 * t) + a * u * math.cos(t) + b * v * math.sin(t)
        step = g / gp if gp > 0 else math.copysign(dt_max, g)
        t -= max(-dt_max, min(dt_max, step))
    d = math.hypot(a * math.cos(t) - u, b * math.sin(t) - v)
    speed = math.hypot(a * math.sin(t), b * math.cos(t))
    return d, 2.0 * math.pi * speed / body["n"]


def fine_integral(body, sigma_b, x, nx, shift, rho):
    """int over the exact curve of `body` (translated by shift) of
    G^t(x, y; nx) sigma^(y) ds_y, sigma^ the trigonometric interpolant of the
    body's nodal density sigma_b (n_b, 2), by the trapezoidal rule on
    rho * n_b points."""
    nb = sigma_b.shape[0]
    nf = rho * nb
    tf = 2.0 * np.pi * np.arange(nf) / nf
    if body.get("shape", "ellipse") == "star":
        yf, dyf, _ = geometry.curve_point(body, tf)
        speed = np.hypot(dyf[:, 0], dyf[:, 1])
    else:
        yf, speed = geometry.ellipse_point(body["a"], body["b"], body["xc"], body["theta"], tf)
    wf = (2.0 * np.pi / nf) * speed
    sf = trig_interp(sigma_b, nf)
    r = np.asarray(x)[None, :] - (yf + np.asarray(shift)[None, :])
    return kernels.traction(r, np.asarray(nx)[None, :], sf * wf[:, None]).sum(0)


class ClosePairs:
    """All (target, source body, image shift) triples closer than
    close_factor * h_b, with the same-body zero-shift case excluded (that
    interaction is the smooth rule plus the on-curve diagonal)."""

    def __init__(self, susp, shifts, close_factor=10.0, targets=None, rule="fine"):
        """targets: restrict the search to these target nodes (None = all).
        rule: "fine" evaluates the integral of the interpolated density by
        the fine trapezoidal rule (its definition); "barycentric" by the
        paper's special quadrature (oracle/barycentric.py)."""
        if rule not in ("fine", "barycentric"):
            raise ValueError("rule is 'fine' or 'barycentric'")
        self.rule = rule
        self.susp = susp
        self.pairs = []  # (target index, body, shift vector, curve distance, local spacing)
        off = susp.offsets
        tidx = np.arange(susp.N) if targets is None else np.asarray(targets)
        for b in range(len(susp.bodies)):
            sl = slice(off[b], off[b + 1])
            yb = susp.x[sl]
            hb = susp.w[sl].sum() / (off[b + 1] - off[b])
            bd = susp.bodies[b]
            for sh in shifts:
                dist = np.sqrt(((susp.x[tidx, None, :] - (yb[None, :, :] + sh)) ** 2).sum(-1))
                d = dist.min(axis=1)
                for row in np.nonzero(d < close_factor * hb)[0]:
                    i = int(tidx[row])
                    if susp.owner[i] == b and sh[0] == 0.0 and sh[1] == 0.0:
                        continue
                    k = int(dist[row].argmin())
                    dc, hl = closest_point(bd, susp.x[i], sh, 2.0 * np.pi * k / bd["n"])
                    self.pairs.append((int(i), b, sh.copy(), dc, hl))

    def apply(self, sigma, targets=None):
        """Correction to the near traction at every target (or the listed
        targets), for the nodal density sigma (N, 2)."""
        susp = self.susp
        want = None if targets is None else {int(t): k for k, t in enumerate(targets)}
        out = np.zeros((susp.N if targets is None else len(targets), 2))
        off = susp.offsets
        for (i, b, sh, d, hl) in self.pairs:
            if want is not None and i not in want:
                continue
            bd = susp.bodies[b]
            sl = slice(off[b], off[b + 1])
            xi = susp.x[i]
            ni = susp.n[i]
            if self.rule == "barycentric":
                from . import barycentric
                fine = barycentric.slp_traction(bd, sigma[sl], xi, ni, sh)
            else:
                fine = fine_integral(bd, sigma[sl], xi, ni, sh, fine_factor(hl, d))
            coarse = kernels.traction(xi[None, :] - (susp.x[sl] + sh), ni[None, :],
                                      sigma[sl] * susp.w[sl, None]).sum(0)
            k = i if want is None else want[i]
            out[k] += fine - coarse
        return out
