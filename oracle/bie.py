"""The discretised mobility BIE and everything around it (oracle, FP64).

Operator, Eq. (BIEdiscretized) with the rigid completion L of Eq.
(BIEPerturbed2) and the pressure fix of the remark "Pressure correction for
GMRES stability" (Sec. 6.2):

  y_i = 1/2 sigma_i + T_i + alpha n_i + F_b + (x_i - x^c_b)^perp tau_b,
  T_i = sum over bodies and 3x3 images of G^t(x_i, y_j; n_i) sigma_j w_j
        (the zero-distance pair replaced by its on-curve limit)
        + proxy correction (Sec. 6.2 step 4) + close correction (Sec. 6.3),
  alpha = -T_0 . n_0 (node 0 of body 0),
  F_b = sum_{j in b} sigma_j w_j,  tau_b = sum_{j in b} (y_j - x^c_b)^perp . sigma_j w_j,

right-hand side -T(u0, p0) = -mu gamma (n_2, n_1) for u0 = (gamma x2, 0),
p0 = 0 and the stress -p I + mu (grad u + grad u^T) of Sec. 3.

Vectors are (N, 2) arrays; the flat form is node-major (x, y interleaved).
"""
import math

import numpy as np

from . import geometry, kernels, periodic
from .close import ClosePairs


def perp(v):
    return np.stack([-v[..., 1], v[..., 0]], axis=-1)


class Operator:
    def __init__(self, susp, n_proxy=16, proxy_radius=1.5, n_coll=16,
                 close_factor=10.0, lam_rel=1e-8, use_close=True, close_targets=None, close_rule="fine"):
        self.s = susp
        self.M = n_proxy
        self.m = n_coll
        self.shifts = periodic.image_shifts(susp.e1, susp.e2)
        self.yp = periodic.proxy_points(susp.centre, proxy_radius, n_proxy)
        self.Q = periodic.proxy_matrix(susp.e1, susp.e2, susp.centre, n_coll, self.yp, susp.mu)
        self.Qp = periodic.proxy_solution_operator(self.Q, lam_rel)
        self.self_index = np.arange(susp.N)
        # close_targets restricts the close-pair search (sampled evaluation of
        # large cells); apply() is then valid at those targets and node 0 only
        # close_rule: "fine" (the definition) or "barycentric" (the paper's Sec. 6.3 rule)
        self.close = ClosePairs(susp, self.shifts, close_factor, close_targets, close_rule) if use_close else None

    # -- pieces ----------------------------------------------------------------
    def density_moments(self, sigma):
        """q = sigma w, per-body net force F_b and torque tau_b (Eq. BIEPerturbed2)."""
        s = self.s
        q = sigma * s.w[:, None]
        nb = len(s.bodies)
        F = np.zeros((nb, 2))
        tau = np.zeros(nb)
        for b in range(nb):
            sl = slice(s.offsets[b], s.offsets[b + 1])
            F[b] = q[sl].sum(0)
            tau[b] = (perp(s.x[sl] - s.xc[b]) * q[sl]).sum()
        return q, F, tau

    def proxy_strengths(self, q):
        s = self.s
        g = periodic.near_discrepancy(s.e1, s.e2, s.centre, self.m, s.x, q, s.mu)
        dt = periodic.corrected_discrepancy(g, q.sum(0), s.e1, s.e2, self.m)
        return periodic.apply_operator_exact(self.Qp, dt), dt

    def traction(self, sigma, targets=None):
        """Periodic traction T (before the pressure fix) at all or listed nodes."""
        s = self.s
        q, _, _ = self.density_moments(sigma)
        idx = np.arange(s.N) if targets is None else np.asarray(targets)
        xt, nt = s.x[idx], s.n[idx]
        T = periodic.near_traction(xt, nt, s.x, q, self.shifts, self_index=idx)
        T += kernels.traction_self(s.kappa[idx], s.tau[idx], q[idx])
        xi, _ = self.proxy_strengths(q)
        T += periodic.correction_traction(xt, nt, self.yp, xi)
        if self.close is not None:
            T += self.close.apply(sigma, None if targets is None else idx)
        return T

    def apply(self, sigma, targets=None):
        """A sigma at all nodes, or at the listed nodes only."""
        s = self.s
        sigma = np.asarray(sigma, dtype=np.float64).reshape(s.N, 2)
        idx = np.arange(s.N) if targets is None else np.asarray(targets)
        want = np.unique(np.concatenate([[0], idx]))
        T = self.traction(sigma, want)
        pos = {int(k): j for j, k in enumerate(want)}
        alpha = -(T[pos[0]] @ s.n[0])
        _, F, tau = self.density_moments(sigma)
        rows = np.array([pos[int(k)] for k in idx])
        b = s.owner[idx]
        y = 0.5 * sigma[idx] + T[rows] + alpha * s.n[idx] + F[b] + perp(s.x[idx] - s.xc[b]) * tau[b][:, None]
        return y

    def matvec(self, v):
        return self.apply(np.asarray(v).reshape(-1, 2)).ravel()

    def rhs(self):
        s = self.s
        return -s.mu * s.gamma * np.stack([s.n[:, 1], s.n[:, 0]], axis=1)

    # -- post-processing --------------------------------------------------------
    def body_velocities(self, sigma):
        """Sec. 3 / Eq. (RigidBodyMotion): inside body b the total flow u + u0
        is the rigid motion v_b + omega_b (x - x^c_b)^perp, so v_b is u + u0 at
        the centroid and omega_b is half the vorticity there.  u is the
        periodic single layer (near sum + proxy velocity), its free constant
        fixed by making the proxy velocity vanish at the cell centre."""
        s = self.s
        sigma = np.asarray(sigma, dtype=np.float64).reshape(s.N, 2)
        q, _, _ = self.density_moments(sigma)
        xi, _ = self.proxy_strengths(q)
        u = periodic.near_velocity(s.xc, s.x, q, self.shifts, s.mu)
        u += periodic.correction_velocity(s.xc, self.yp, xi, s.mu)
        u -= periodic.correction_velocity(s.centre[None, :], self.yp, xi, s.mu)
        w = periodic.near_vorticity(s.xc, s.x, q, self.shifts, s.mu)
        w += periodic.correction_vorticity(s.xc, self.yp, xi, s.mu)
        v = u + np.stack([s.gamma * s.xc[:, 1], np.zeros(len(s.bodies))], axis=1)
        omega = 0.5 * (w - s.gamma)
        return v, omega

    def mu_eff(self, sigma):
        """Effective viscosity as the particle-stress (stresslet) cell average:
        mu_eff = mu - (1/(gamma |U|)) sum_b int_{Gamma_b} (x_2 - x^c_2) sigma_1 ds.
        The exterior traction of u + u0 is -sigma (jump of Lemma
        jumprelation with zero interior traction)."""
        s = self.s
        sigma = np.asarray(sigma, dtype=np.float64).reshape(s.N, 2)
        dy = s.x[:, 1] - s.xc[s.owner, 1]
        return s.mu - (sigma[:, 0] * dy * s.w).sum() / (s.gamma * s.cell_area)

    def mu_eff_wall(self, sigma, m_wall=64):
        """Eq. (mueff): shear force through the bottom wall D per unit shear,
        valid when no body meets D (used to pin mu_eff)."""
        s = self.s
        sigma = np.asarray(sigma, dtype=np.float64).reshape(s.N, 2)
        q, _, _ = self.density_moments(sigma)
        xi, _ = self.proxy_strengths(q)
        sgl, wgl = periodic.gauss_legendre_unit(m_wall)
        xd = s.centre[None, :] - 0.5 * s.e2[None, :] + sgl[:, None] * s.e1[None, :]
        nD = np.repeat(np.array([[0.0, 1.0]]), m_wall, axis=0)
        T = periodic.near_traction(xd, nD, s.x, q, self.shifts)
        T += periodic.correction_traction(xd, nD, self.yp, xi)
        t1 = T[:, 0] + s.mu * s.gamma
        return (t1 * wgl).sum() * np.hypot(*s.e1) / (s.gamma * np.hypot(*s.e1))


# ----------------------------------------------------------------------------
# GMRES (unrestarted Arnoldi with modified Gram-Schmidt, Givens rotations)
# ----------------------------------------------------------------------------
def gmres(matvec, b, tol=1e-10, maxiter=500, x0=None):
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - matvec(x) if x0 is not None else b.copy()
    bnorm = np.linalg.norm(b)
    beta = np.linalg.norm(r)
    hist = [beta / bnorm]
    if beta <= tol * bnorm:
        return x, 0, hist
    m = min(maxiter, n)
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    cs, sn = np.zeros(m), np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    V[0] = r / beta
    k = 0
    for k in range(m):
        w = matvec(V[k])
        for j in range(k + 1):
            H[j, k] = V[j] @ w
            w = w - H[j, k] * V[j]
        H[k + 1, k] = np.linalg.norm(w)
        if H[k + 1, k] > 0:
            V[k + 1] = w / H[k + 1, k]
        for j in range(k):
            h0 = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
            H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
            H[j, k] = h0
        den = math.hypot(H[k, k], H[k + 1, k])
        cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
        H[k, k] = den
        H[k + 1, k] = 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        hist.append(abs(g[k + 1]) / bnorm)
        if abs(g[k + 1]) <= tol * bnorm:
            break
    kk = k + 1
    yk = np.linalg.solve(np.triu(H[:kk, :kk]), g[:kk])
    x = x + V[:kk].T @ yk
    return x, kk, hist


def solve(op, b=None, tol=1e-10, maxiter=500, x0=None, max_restarts=5):
    """GMRES to a true relative residual ||b - A x|| / ||b|| <= tol."""
    b = op.rhs().ravel() if b is None else np.asarray(b, dtype=np.float64).ravel()
    x = None if x0 is None else np.asarray(x0, dtype=np.float64).ravel()
    total = 0
    for _ in range(max_restarts):
        x, it, _ = gmres(op.matvec, b, tol, maxiter, x)
        total += it
        res = np.linalg.norm(b - op.matvec(x)) / np.linalg.norm(b)
        if res <= tol:
            break
    return x.reshape(-1, 2), total, res


# ----------------------------------------------------------------------------
# time stepping (Sec. 7)
# ----------------------------------------------------------------------------
def euler_step(susp, e2_0, t, dt, op_kwargs, sigma0=None, tol=1e-10, operator=None):
    """One forward-Euler step s <- s + dt F(t, s).  Returns the new
    Suspension, the new time, and (sigma, v, omega, mu_eff) at time t.
    operator: the Operator class to build (a subclass that evaluates the same
    matvec in parallel, say); Operator by default."""
    op = (operator or Operator)(susp, **op_kwargs)
    sigma, iters, res = solve(op, tol=tol, x0=sigma0)
    v, omega = op.body_velocities(sigma)
    mu_eff = op.mu_eff(sigma)
    t1 = t + dt
    e1, e2 = geometry.lattice_at(susp.e1, e2_0, susp.gamma, t1)
    bodies = []
    for b, bd in enumerate(susp.bodies):
        nb = dict(bd)
        xc = np.asarray(bd["xc"]) + dt * v[b]
        nb["xc"] = geometry.wrap_into_cell(xc, e1, e2, susp.centre)
        nb["theta"] = bd["theta"] + dt * omega[b]
        bodies.append(nb)
    new = geometry.Suspension(e1, e2, susp.centre, susp.mu, susp.gamma, bodies)
    return new, t1, dict(sigma=sigma, v=v, omega=omega, mu_eff=mu_eff, iters=iters, res=res)


# ----------------------------------------------------------------------------
# the paper's own periodizer, as an independent check of the 3 x 3 reading
# ----------------------------------------------------------------------------
class OperatorUtilde(Operator):
    """The same BIE operator with the paper's periodizer (Def. Gnear, remark
    after Eq. W): each source node contributes its four lattice images inside
    the doubled cell U~, chosen per node by its lattice coordinates, and the
    proxies sit on the walls of U~ (periodic.proxy_points_box).  The
    periodic sums of Sec. 6.2 are evaluated at targets in the unit cell U: a
    node outside U (on a body across a wall) is evaluated at its lattice
    translate inside U, where the periodic traction takes the same value
    (with the node's own normal); its self pair is the image of itself
    that lands there.  The wall discrepancy takes the cancellation form of
Sec. 6.2 step 2 (periodic.near_discrepancy_utilde), so that no evaluation
comes near a body that crosses a wall.  Both
    periodizers define the same periodic Green's function up to constants,
    so densities, rotation rates and mu_eff agree to discretisation accuracy.

    Close evaluation (Sec. 6.3) is the 3 x 3 operator's, pair for pair, in
    the nodes' own frame: a pair (target, body, image) is valid here when
    every node of the body has that image, seen from the target's translate
    inside U, among its four; with bodies smaller than about half a cell
    this always holds (images left out lie at least half a cell from U), and
    a geometry where it does not is refused (ValueError)."""

    def __init__(self, susp, n_proxy=128, n_coll=32, lam_rel=1e-8, close_factor=10.0, use_close=True,
                 close_targets=None, close_rule="fine"):
        self.s = susp
        self.M = n_proxy
        self.m = n_coll
        self.yp = periodic.proxy_points_box(susp.e1, susp.e2, susp.centre, n_proxy)
        self.Q = periodic.proxy_matrix(susp.e1, susp.e2, susp.centre, n_coll, self.yp, susp.mu)
        self.Qp = periodic.proxy_solution_operator(self.Q, lam_rel)
        self.imgmn = periodic.utilde_images(susp.e1, susp.e2, susp.centre, susp.x)
        self.img = periodic.utilde_shifts(susp.e1, susp.e2, susp.centre, susp.x)
        self.wrapmn = periodic.wrap_images(susp.e1, susp.e2, susp.centre, susp.x)
        self.wrap = self.wrapmn[:, :1] * susp.e1[None, :] + self.wrapmn[:, 1:] * susp.e2[None, :]
        # the copy of node i at its translate inside U (index into the expanded sources)
        hit = np.all(self.imgmn == self.wrapmn[:, None, :], axis=2)
        assert hit.sum(axis=1).min() == 1
        self.own_wrapped = np.arange(susp.N) * 4 + hit.argmax(axis=1)
        self.zero = [np.zeros(2)]
        self.close = None
        if use_close:
            shifts = periodic.image_shifts(susp.e1, susp.e2)
            self.close = ClosePairs(susp, shifts, close_factor, close_targets, close_rule)
            E = np.column_stack([susp.e1, susp.e2])
            for (i, b, sh, _, _) in self.close.pairs:
                mn = np.rint(np.linalg.solve(E, sh)).astype(np.int64) + self.wrapmn[i]
                sl = slice(susp.offsets[b], susp.offsets[b + 1])
                if not np.all(np.any(np.all(self.imgmn[sl] == mn[None, None, :], axis=2), axis=1)):
                    raise ValueError("a close pair's body image is not wholly among the doubled-cell images "
                                     "(a body larger than about half a cell?)")

    def _sources(self, q):
        return periodic.expand_images(self.s.x, q, self.img)

    def targets(self, idx):
        """Translates inside U of the listed nodes."""
        return self.s.x[idx] + self.wrap[idx]

    def proxy_strengths(self, q):
        s = self.s
        g = periodic.near_discrepancy_utilde(s.e1, s.e2, s.centre, self.m, s.x, q, self.imgmn, s.mu)
        dt = periodic.corrected_discrepancy(g, q.sum(0), s.e1, s.e2, self.m)
        return periodic.apply_operator_exact(self.Qp, dt), dt

    def traction(self, sigma, targets=None):
        s = self.s
        q, _, _ = self.density_moments(sigma)
        idx = np.arange(s.N) if targets is None else np.asarray(targets)
        Y, Q, _ = self._sources(q)
        xt = self.targets(idx)
        T = periodic.near_traction(xt, s.n[idx], Y, Q, self.zero, self_index=self.own_wrapped[idx])
        T += kernels.traction_self(s.kappa[idx], s.tau[idx], q[idx])
        xi, _ = self.proxy_strengths(q)
        T += periodic.correction_traction(xt, s.n[idx], self.yp, xi)
        if self.close is not None:
            T += self.close.apply(sigma, None if targets is None else idx)
        return T

    def body_velocities(self, sigma):
        s = self.s
        sigma = np.asarray(sigma, dtype=np.float64).reshape(s.N, 2)
        q, _, _ = self.density_moments(sigma)
        xi, _ = self.proxy_strengths(q)
        Y, Q, _ = self._sources(q)
        u = periodic.near_velocity(s.xc, Y, Q, self.zero, s.mu)
        u += periodic.correction_velocity(s.xc, self.yp, xi, s.mu)
        u -= periodic.correction_velocity(s.centre[None, :], self.yp, xi, s.mu)
        w = periodic.near_vorticity(s.xc, Y, Q, self.zero, s.mu)
        w += periodic.correction_vorticity(s.xc, self.yp, xi, s.mu)
        v = u + np.stack([s.gamma * s.xc[:, 1], np.zeros(len(s.bodies))], axis=1)
        omega = 0.5 * (w - s.gamma)
        return v, omega

    def mu_eff_contour(self, sigma, m_wall=32):
        """Sec. 6.4 (Eq. contourdef): mu_eff from the shear force through a
        contour C that runs from L to R below every body, with no quadrature
        near any curve.  The curve splits into quadrant pieces by lattice
        coordinates (1: s >= 0, t >= 0; 2: s < 0, t >= 0; 3: s < 0, t < 0;
        4: s >= 0, t < 0) and Gamma~ = {Gamma_1 - e1 - e2, Gamma_2 - e2,
        Gamma_3, Gamma_4 - e1}, so that this periodizer's near sum at x is the
        potential of Gamma~ at x, x - e1, x - e2 and x - e1 - e2.  Gauss' law
        (exterior traction integral = -sum of the enclosed forces, outward
        normals) on the boundary of the two cells below U gives
            int_C T = 2 int_{D-e2} S~ + 2 int_{D-e1-e2} S~ + int_{R-e2} S~
                      - int_{L-e1-e2} S~ - sum_{Gamma_1, Gamma_2} q + int_D T(v, q)
        with the normal (0, 1) on D and the outward normal of L on L and R
        (reading 2), the signs the paper prints.  (Its printed Gamma~ names
        Gamma_1 in place of Gamma_2 and Gamma_4 in two pieces; the shifts
        above are the ones that reproduce the near sum.)"""
        s = self.s
        sigma = np.asarray(sigma, dtype=np.float64).reshape(s.N, 2)
        q, _, _ = self.density_moments(sigma)
        xi, _ = self.proxy_strengths(q)
        e1, e2, c = s.e1, s.e2, s.centre
        st = np.linalg.solve(np.column_stack([e1, e2]), (s.x - c).T).T
        right, up = st[:, 0] >= 0, st[:, 1] >= 0
        shift = np.where(right[:, None], -e1[None, :], 0.0) + np.where(up[:, None], -e2[None, :], 0.0)
        yt = s.x + shift  # Gamma~
        zero = [np.zeros(2)]
        gl, wl = periodic.gauss_legendre_unit(m_wall)
        nl, _ = periodic.wall_normals(e1, e2)
        nD = np.array([0.0, 1.0])

        def wall_int(start, along, normal):
            xw = start[None, :] + gl[:, None] * along[None, :]
            nw = np.repeat(normal[None, :], m_wall, axis=0)
            T = periodic.near_traction(xw, nw, yt, q, zero)
            return (T * wl[:, None]).sum(0) * np.hypot(*along)

        d_e2 = c - 1.5 * e2            # midpoint of D - e2
        d_e1e2 = c - e1 - 1.5 * e2     # D - e1 - e2
        r_e2 = c + 0.5 * e1 - e2       # R - e2
        l_e1e2 = c - 1.5 * e1 - e2     # L - e1 - e2
        F = (2 * wall_int(d_e2, e1, nD) + 2 * wall_int(d_e1e2, e1, nD)
             + wall_int(r_e2, e2, nl) - wall_int(l_e1e2, e2, nl) - q[up].sum(0))
        xd = c[None, :] - 0.5 * e2[None, :] + gl[:, None] * e1[None, :]
        Tv = periodic.correction_traction(xd, np.repeat(nD[None, :], m_wall, axis=0), self.yp, xi)
        F += (Tv * wl[:, None]).sum(0) * np.hypot(*e1)
        l1 = np.hypot(*e1)
        return s.mu + F[0] / (s.gamma * l1)
