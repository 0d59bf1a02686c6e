"""Boundary discretisation and lattice geometry (oracle, FP64).

Sec. 6 (opening): on a 2*pi-periodic parametrisation x(t) the periodic
trapezoidal rule takes nodes x(2*pi*k/N) and weights (2*pi/N)*|x'(2*pi*k/N)|.
Sec. 2: the centroid x^c of a body is the arc-length mean of its boundary; for
an ellipse it is the ellipse centre.  Sec. 7: e1 = (1, 0) and
e2(t) = (gamma*t - round(gamma*t), 1), round = nearest integer.
"""
import math

import numpy as np


def ellipse_nodes(a, b, centre, theta, n):
    """Nodes of the ellipse centre + R(theta) (a cos t, b sin t), t = 2*pi*k/n.

    Returns a dict with
      x      (n, 2) node positions,
      tau    (n, 2) unit tangent (counter-clockwise),
      n      (n, 2) outward unit normal (tangent turned clockwise),
      w      (n,)   trapezoidal weights (2*pi/n)*|x'|,
      kappa  (n,)   signed curvature (positive for a convex CCW curve),
      t      (n,)   parameter values.
    """
    t = 2.0 * np.pi * np.arange(n) / n
    c, s = math.cos(theta), math.sin(theta)
    rot = np.array([[c, -s], [s, c]])
    p = np.stack([a * np.cos(t), b * np.sin(t)], axis=1)
    dp = np.stack([-a * np.sin(t), b * np.cos(t)], axis=1)
    ddp = -p
    x = np.asarray(centre, dtype=np.float64)[None, :] + p @ rot.T
    dx = dp @ rot.T
    ddx = ddp @ rot.T
    speed = np.hypot(dx[:, 0], dx[:, 1])
    tau = dx / speed[:, None]
    nrm = np.stack([tau[:, 1], -tau[:, 0]], axis=1)
    w = (2.0 * np.pi / n) * speed
    kappa = (dx[:, 0] * ddx[:, 1] - dx[:, 1] * ddx[:, 0]) / speed**3
    return dict(x=x, tau=tau, n=nrm, w=w, kappa=kappa, t=t)


def star_radius(r0, eps, k, t):
    """Polar radius r(t) = r0 (1 + eps cos(k t)) of a star-shaped body and its
    first two derivatives in t (Sec. 8 Examples 4-5: x(t) = (r(t) cos t,
    r(t) sin t) about the centre)."""
    t = np.asarray(t, dtype=np.float64)
    r = r0 * (1.0 + eps * np.cos(k * t))
    dr = -r0 * eps * k * np.sin(k * t)
    ddr = -r0 * eps * k * k * np.cos(k * t)
    return r, dr, ddr


def curve_point(body, t):
    """Point, first and second derivative in t of a body's boundary
    x(t) = x^c + R(theta) p(t): an ellipse p = (a cos t, b sin t), or a star
    p = r(t) (cos t, sin t) (body["shape"] == "star": r0, eps, k).  Returns
    three (len(t), 2) arrays."""
    t = np.asarray(t, dtype=np.float64)
    if body.get("shape", "ellipse") == "star":
        r, dr, ddr = star_radius(body["r0"], body["eps"], body["k"], t)
        c_, s_ = np.cos(t), np.sin(t)
        p = np.stack([r * c_, r * s_], axis=1)
        dp = np.stack([dr * c_ - r * s_, dr * s_ + r * c_], axis=1)
        ddp = np.stack([ddr * c_ - 2 * dr * s_ - r * c_, ddr * s_ + 2 * dr * c_ - r * s_], axis=1)
    else:
        a, b = body["a"], body["b"]
        p = np.stack([a * np.cos(t), b * np.sin(t)], axis=1)
        dp = np.stack([-a * np.sin(t), b * np.cos(t)], axis=1)
        ddp = -p
    c, s = math.cos(body["theta"]), math.sin(body["theta"])
    rot = np.array([[c, -s], [s, c]])
    return np.asarray(body["xc"], dtype=np.float64)[None, :] + p @ rot.T, dp @ rot.T, ddp @ rot.T


def body_nodes(body):
    """Trapezoidal discretisation of any body (as ellipse_nodes)."""
    n = body["n"]
    t = 2.0 * np.pi * np.arange(n) / n
    x, dx, ddx = curve_point(body, t)
    speed = np.hypot(dx[:, 0], dx[:, 1])
    tau = dx / speed[:, None]
    nrm = np.stack([tau[:, 1], -tau[:, 0]], axis=1)
    w = (2.0 * np.pi / n) * speed
    kappa = (dx[:, 0] * ddx[:, 1] - dx[:, 1] * ddx[:, 0]) / speed**3
    return dict(x=x, tau=tau, n=nrm, w=w, kappa=kappa, t=t)


def body_radius(body):
    """Largest distance from the centre to the boundary."""
    if body.get("shape", "ellipse") == "star":
        return body["r0"] * (1.0 + abs(body["eps"]))
    return max(body["a"], body["b"])


def ellipse_point(a, b, centre, theta, t):
    """Position and speed on the exact ellipse at parameter values t."""
    t = np.asarray(t, dtype=np.float64)
    c, s = math.cos(theta), math.sin(theta)
    px, py = a * np.cos(t), b * np.sin(t)
    dpx, dpy = -a * np.sin(t), b * np.cos(t)
    x = np.stack([centre[0] + c * px - s * py, centre[1] + s * px + c * py], axis=1)
    dx = np.stack([c * dpx - s * dpy, s * dpx + c * dpy], axis=1)
    return x, np.hypot(dx[:, 0], dx[:, 1])


def round_half_away(v):
    """round() as in C: nearest integer, halves away from zero (Sec. 7)."""
    return math.copysign(math.floor(abs(v) + 0.5), v)


def lattice_at(e1, e2_0, gamma, t):
    """Sec. 7: the lattice sheared by rate gamma for time t, skew kept bounded.

    e1 = (L1, 0) stays fixed; the top of the cell moves with the background
    shear u0 = (gamma*x2, 0), so e2 gains gamma*t*L2 in x, and is reduced by
    the integer multiple of e1 nearest to its x component.
    """
    e1 = np.asarray(e1, dtype=np.float64)
    e2_0 = np.asarray(e2_0, dtype=np.float64)
    if e1[1] != 0.0:
        raise ValueError("time stepping expects e1 = (L1, 0)")
    sx = e2_0[0] + gamma * t * e2_0[1]
    sx -= e1[0] * round_half_away(sx / e1[0])
    return e1.copy(), np.array([sx, e2_0[1]])


def wrap_into_cell(p, e1, e2, centre):
    """Translate p by a lattice vector so that its lattice coordinates about
    the cell centre lie in [-1/2, 1/2)."""
    mat = np.array([[e1[0], e2[0]], [e1[1], e2[1]]])
    ab = np.linalg.solve(mat, np.asarray(p, dtype=np.float64) - centre)
    shift = np.floor(ab + 0.5)
    return np.asarray(p, dtype=np.float64) - mat @ shift


class Suspension:
    """One unit cell: lattice, fluid, and a list of ellipses.

    bodies: list of dicts with keys xc (2,), theta, n and the shape: a, b
    (ellipse), or shape = "star" with r0, eps, k (r(t) = r0 (1 + eps cos kt)).
    The centre xc is the reference point of the rigid motion (for an ellipse
    and a star with k >= 2 also the boundary's arc-length centroid).
    """

    def __init__(self, e1, e2, centre, mu, gamma, bodies):
        self.e1 = np.asarray(e1, dtype=np.float64)
        self.e2 = np.asarray(e2, dtype=np.float64)
        self.centre = np.asarray(centre, dtype=np.float64)
        self.mu = float(mu)
        self.gamma = float(gamma)
        self.bodies = [dict(b) for b in bodies]
        self.discretise()

    def discretise(self):
        xs, taus, ns, ws, ks, ts, owner = [], [], [], [], [], [], []
        offsets = [0]
        for i, bd in enumerate(self.bodies):
            g = (body_nodes(bd) if bd.get("shape", "ellipse") == "star"
                 else ellipse_nodes(bd["a"], bd["b"], bd["xc"], bd["theta"], bd["n"]))
            xs.append(g["x"])
            taus.append(g["tau"])
            ns.append(g["n"])
            ws.append(g["w"])
            ks.append(g["kappa"])
            ts.append(g["t"])
            owner.append(np.full(bd["n"], i))
            offsets.append(offsets[-1] + bd["n"])
        self.x = np.concatenate(xs)
        self.tau = np.concatenate(taus)
        self.n = np.concatenate(ns)
        self.w = np.concatenate(ws)
        self.kappa = np.concatenate(ks)
        self.t = np.concatenate(ts)
        self.owner = np.concatenate(owner)
        self.offsets = np.array(offsets)
        self.xc = np.array([bd["xc"] for bd in self.bodies], dtype=np.float64).reshape(-1, 2)
        self.N = int(self.offsets[-1])

    @property
    def cell_area(self):
        return abs(self.e1[0] * self.e2[1] - self.e1[1] * self.e2[0])
