"""Periodized sums (oracle, FP64): Sec. 4.2 and Sec. 6.1-6.2.

The periodic single-layer traction at a target is split (Eq. GperDecomp,
Eq. Stsplit) into
  * a NEAR image sum of free-space kernels over the 3 x 3 block of lattice
    translates m e1 + n e2, m, n in {-1, 0, 1}, of every source, and
  * a CORRECTION: the solution of the empty-box BVP (Eqs. emptyBoxEq1-4)
    whose wall discrepancy cancels that of the near sum and adds the net-force
    traction jumps F/(2|e2|) on L-R and F/(2|e1|) on D-U (Eqs.
    SLPdiscrepCorr1-4, algorithm of Sec. 6.2 step 3), represented by M proxy
    Stokeslets (Eq. vrep) fitted by least squares at Gauss-Legendre
    collocation points on the walls L and D (Sec. 6.1).

Wall normal convention (fixed by the consistency computation of App. B): the
traction on L and R is taken with the outward normal of L, and on D and U with
the outward normal of D, so that int_L g2 + int_D g4 = 0 holds for any net
force (Eq. gforce).
"""
import numpy as np

from . import kernels

IMAGES_3x3 = [(m, n) for n in (-1, 0, 1) for m in (-1, 0, 1)]


def image_shifts(e1, e2, images=IMAGES_3x3):
    return [m * e1 + n * e2 for (m, n) in images]


# ----------------------------------------------------------------------------
# direct sums
# ----------------------------------------------------------------------------
def near_traction(xt, nt, ys, qs, shifts, self_index=None, chunk=256):
    """sum_shift sum_j G^t(x_i, y_j + shift; n_i) q_j  (Sec. 6.2 step 1).

    self_index[i] = j marks source j as the same point as target i; that pair
    is skipped for the zero shift (the caller adds the on-curve limit).
    """
    xt = np.atleast_2d(xt)
    out = np.zeros_like(xt)
    for s0 in range(0, xt.shape[0], chunk):
        sl = slice(s0, s0 + chunk)
        acc = np.zeros_like(xt[sl])
        for sh in shifts:
            r = xt[sl, None, :] - (ys[None, :, :] + sh[None, None, :])
            if self_index is not None and sh[0] == 0.0 and sh[1] == 0.0:
                mask = self_index[sl, None] == np.arange(ys.shape[0])[None, :]
                r = np.where(mask[..., None], 1.0, r)
                contrib = kernels.traction(r, nt[sl, None, :], qs[None, :, :])
                contrib = np.where(mask[..., None], 0.0, contrib)
            else:
                contrib = kernels.traction(r, nt[sl, None, :], qs[None, :, :])
            acc += contrib.sum(axis=1)
        out[sl] = acc
    return out


def near_velocity(xt, ys, qs, shifts, mu, chunk=256):
    """sum_shift sum_j G(x_i, y_j + shift) q_j."""
    xt = np.atleast_2d(xt)
    out = np.zeros_like(xt)
    for s0 in range(0, xt.shape[0], chunk):
        sl = slice(s0, s0 + chunk)
        acc = np.zeros_like(xt[sl])
        for sh in shifts:
            r = xt[sl, None, :] - (ys[None, :, :] + sh[None, None, :])
            acc += kernels.stokeslet(r, qs[None, :, :], mu).sum(axis=1)
        out[sl] = acc
    return out


def near_vorticity(xt, ys, qs, shifts, mu):
    xt = np.atleast_2d(xt)
    acc = np.zeros(xt.shape[0])
    for sh in shifts:
        r = xt[:, None, :] - (ys[None, :, :] + sh[None, None, :])
        acc += kernels.stokeslet_vorticity(r, qs[None, :, :], mu).sum(axis=1)
    return acc


# ----------------------------------------------------------------------------
# walls, collocation and proxies (Sec. 6.1)
# ----------------------------------------------------------------------------
def gauss_legendre_unit(m):
    """m Gauss-Legendre nodes on (-1/2, 1/2) and weights summing to 1."""
    s, w = np.polynomial.legendre.leggauss(m)
    return 0.5 * s, 0.5 * w


def wall_normals(e1, e2):
    """Unit outward normals of the walls L (parallel to e2) and D (parallel
    to e1): nu_L is orthogonal to e2 with nu_L . e1 < 0, nu_D is orthogonal
    to e1 with nu_D . e2 < 0."""
    nl = np.array([e2[1], -e2[0]]) / np.hypot(*e2)
    if nl @ e1 > 0:
        nl = -nl
    nd = np.array([e1[1], -e1[0]]) / np.hypot(*e1)
    if nd @ e2 > 0:
        nd = -nd
    return nl, nd


def collocation(e1, e2, centre, m):
    """Collocation points on L = {c - e1/2 + s e2} and D = {c - e2/2 + s e1},
    s at Gauss-Legendre nodes of (-1/2, 1/2); with arc-length weights."""
    s, w = gauss_legendre_unit(m)
    xl = centre[None, :] - 0.5 * e1[None, :] + s[:, None] * e2[None, :]
    xd = centre[None, :] - 0.5 * e2[None, :] + s[:, None] * e1[None, :]
    return xl, xd, w * np.hypot(*e2), w * np.hypot(*e1)


def proxy_points(centre, radius, M):
    ang = 2.0 * np.pi * np.arange(M) / M
    return centre[None, :] + radius * np.stack([np.cos(ang), np.sin(ang)], axis=1)


def _split(v):
    """(m, 2) -> [all 1-components; all 2-components] (Sec. 6.1 ordering)."""
    return np.concatenate([v[:, 0], v[:, 1]])


def proxy_matrix(e1, e2, centre, m, yp, mu):
    """Q = [Q1; Q2; Q3; Q4] (8m x 2M): discrepancies on the walls of the unit
    proxy Stokeslets (Sec. 6.1).  Columns: xi_1 of every proxy, then xi_2."""
    xl, xd, _, _ = collocation(e1, e2, centre, m)
    nl, nd = wall_normals(e1, e2)
    M = yp.shape[0]
    Q = np.zeros((8 * m, 2 * M))
    for comp in range(2):
        f = np.zeros((M, 2))
        f[:, comp] = 1.0
        for p in range(M):
            fp = f[p]
            def vel(x):
                return kernels.stokeslet(x - yp[p], fp[None, :], mu)
            def trac(x, nu):
                return kernels.traction(x - yp[p], nu[None, :], fp[None, :])
            col = comp * M + p
            Q[0 * m:2 * m, col] = _split(vel(xl + e1) - vel(xl))
            Q[2 * m:4 * m, col] = _split(trac(xl + e1, nl) - trac(xl, nl))
            Q[4 * m:6 * m, col] = _split(vel(xd + e2) - vel(xd))
            Q[6 * m:8 * m, col] = _split(trac(xd + e2, nd) - trac(xd, nd))
    return Q


def consistency_matrix(e1, e2, centre, m):
    """W^T (3 x 8m) of Eq. (W), read as the discrete Eqs. (gforce), (gvol):
    rows 1-2 integrate g2 over L plus g4 over D (net force), row 3 integrates
    the normal flux g1 . nu_L over L plus g3 . nu_D over D (volume)."""
    _, _, wl, wd = collocation(e1, e2, centre, m)
    nl, nd = wall_normals(e1, e2)
    z = np.zeros(m)
    W = np.zeros((3, 8 * m))
    W[0] = np.concatenate([z, z, wl, z, z, z, wd, z])
    W[1] = np.concatenate([z, z, z, wl, z, z, z, wd])
    W[2] = np.concatenate([wl * nl[0], wl * nl[1], z, z, wd * nd[0], wd * nd[1], z, z])
    return W


def near_discrepancy(e1, e2, centre, m, ys, qs, mu):
    """g = [g1; g2; g3; g4] of the near sum (Sec. 6.2 step 2), using the
    translation invariance of the kernels: of the 3 x 3 images only the
    columns m = -2 (seen from R, i.e. shifted) and m = +1 survive in
    S_near(x + e1) - S_near(x), and likewise rows for U - D, so every
    evaluation is at least about one cell width from its source."""
    xl, xd, _, _ = collocation(e1, e2, centre, m)
    nl, nd = wall_normals(e1, e2)
    plus_lr = [-2 * e1 + n * e2 for n in (-1, 0, 1)]
    minus_lr = [e1 + n * e2 for n in (-1, 0, 1)]
    plus_du = [k * e1 - 2 * e2 for k in (-1, 0, 1)]
    minus_du = [k * e1 + e2 for k in (-1, 0, 1)]
    nlm = np.repeat(nl[None, :], m, axis=0)
    ndm = np.repeat(nd[None, :], m, axis=0)
    g1 = near_velocity(xl, ys, qs, plus_lr, mu) - near_velocity(xl, ys, qs, minus_lr, mu)
    g2 = near_traction(xl, nlm, ys, qs, plus_lr) - near_traction(xl, nlm, ys, qs, minus_lr)
    g3 = near_velocity(xd, ys, qs, plus_du, mu) - near_velocity(xd, ys, qs, minus_du, mu)
    g4 = near_traction(xd, ndm, ys, qs, plus_du) - near_traction(xd, ndm, ys, qs, minus_du)
    return np.concatenate([_split(g1), _split(g2), _split(g3), _split(g4)])


def near_discrepancy_direct(e1, e2, centre, m, ys, qs, mu):
    """The same g computed literally as S_near(R) - S_near(L) etc. with the
    full 3 x 3 sums (used only to pin the cancellation form)."""
    xl, xd, _, _ = collocation(e1, e2, centre, m)
    nl, nd = wall_normals(e1, e2)
    sh = image_shifts(e1, e2)
    nlm = np.repeat(nl[None, :], m, axis=0)
    ndm = np.repeat(nd[None, :], m, axis=0)
    g1 = near_velocity(xl + e1, ys, qs, sh, mu) - near_velocity(xl, ys, qs, sh, mu)
    g2 = near_traction(xl + e1, nlm, ys, qs, sh) - near_traction(xl, nlm, ys, qs, sh)
    g3 = near_velocity(xd + e2, ys, qs, sh, mu) - near_velocity(xd, ys, qs, sh, mu)
    g4 = near_traction(xd + e2, ndm, ys, qs, sh) - near_traction(xd, ndm, ys, qs, sh)
    return np.concatenate([_split(g1), _split(g2), _split(g3), _split(g4)])


def corrected_discrepancy(g, F, e1, e2, m):
    """g~ = g0 - g with g0 = [0; F/(2|e2|); 0; F/(2|e1|)] (Sec. 6.2 step 3)."""
    g0 = np.zeros(8 * m)
    l2, l1 = np.hypot(*e2), np.hypot(*e1)
    g0[2 * m:3 * m] = F[0] / (2 * l2)
    g0[3 * m:4 * m] = F[1] / (2 * l2)
    g0[6 * m:7 * m] = F[0] / (2 * l1)
    g0[7 * m:8 * m] = F[1] / (2 * l1)
    return g0 - g


def proxy_solution_operator(Q, lam_rel=1e-8):
    """Solution operator P (2M x 8m) of the least-squares fit Q xi = d of
    Sec. 6.1, xi = P d.  Q is rectangular and ill-conditioned (Sec. 6.1), so
    "least squares" is read as the Tikhonov-regularised problem
        min |Q xi - d|^2 + lam^2 |xi|^2,   lam = lam_rel * ||Q||_F,
    whose solution is unique and depends smoothly on Q.  It is obtained here
    from numpy's least-squares solver on the stacked system [Q; lam I]."""
    lam = lam_rel * np.linalg.norm(Q)
    k, n = Q.shape
    A = np.vstack([Q, lam * np.eye(n)])
    B = np.vstack([np.eye(k), np.zeros((n, k))])
    return np.linalg.lstsq(A, B, rcond=None)[0]


def _two_prod(a, b):
    """a*b = p + e exactly (Dekker's product with Veltkamp splitting)."""
    p = a * b
    f = 134217729.0  # 2^27 + 1
    def split(x):
        c = f * x
        hi = c - (c - x)
        return hi, x - hi
    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def apply_operator_exact(P, d):
    """xi = P d with every row summed exactly and rounded once (exact
    products by _two_prod, math.fsum over them), so that the application of
    the fixed proxy operator adds no rounding noise beyond the final rounding
    (P has entries up to ~1/lam, and a plain double-precision product would
    add noise of relative size ~1e-11 to the correction)."""
    import math
    p, e = _two_prod(P, d[None, :])
    return np.array([math.fsum(np.concatenate([p[r], e[r]])) for r in range(P.shape[0])])


def xi_pairs(xi):
    M = xi.shape[0] // 2
    return np.stack([xi[:M], xi[M:]], axis=1)


def correction_traction(xt, nt, yp, xi):
    """T(v, q) at targets of the proxy representation, Eqs. (vrep), (qrep)."""
    f = xi_pairs(xi)
    r = np.atleast_2d(xt)[:, None, :] - yp[None, :, :]
    return kernels.traction(r, np.atleast_2d(nt)[:, None, :], f[None, :, :]).sum(axis=1)


def correction_velocity(xt, yp, xi, mu):
    f = xi_pairs(xi)
    r = np.atleast_2d(xt)[:, None, :] - yp[None, :, :]
    return kernels.stokeslet(r, f[None, :, :], mu).sum(axis=1)


def correction_vorticity(xt, yp, xi, mu):
    f = xi_pairs(xi)
    r = np.atleast_2d(xt)[:, None, :] - yp[None, :, :]
    return kernels.stokeslet_vorticity(r, f[None, :, :], mu).sum(axis=1)


def proxy_points_box(e1, e2, centre, M):
    """The paper's own proxy placement (Sec. 6.1, remark after Eq. W): M
    points on the walls of the doubled cell U~ (walls at lattice coordinate
    +-1), M/4 per wall at the midpoints of equal sub-intervals."""
    k = M // 4
    s = (np.arange(k) + 0.5) / k * 2.0 - 1.0
    pts = []
    for side in (-1.0, 1.0):
        pts.append(centre[None, :] + side * e1[None, :] + s[:, None] * e2[None, :])
        pts.append(centre[None, :] + side * e2[None, :] + s[:, None] * e1[None, :])
    return np.concatenate(pts)


# ----------------------------------------------------------------------------
# the paper's own periodizer (Def. Gnear): per-source images inside U~
# ----------------------------------------------------------------------------
def lattice_coords(e1, e2, centre, ys):
    """(s, t) with y - centre = s e1 + t e2, per point (N, 2)."""
    E = np.column_stack([e1, e2])
    return np.linalg.solve(E, (np.asarray(ys) - centre).T).T


def utilde_images(e1, e2, centre, ys):
    """Per source point the integer pairs (m, n) of the four lattice
    translates y + m e1 + n e2 inside the doubled cell U~ (same centre as U,
    walls at lattice coordinates -1 and +1, Def. Gnear): with (s, t) the
    lattice coordinates of y - centre, m runs over the two integers with
    -1 <= s + m < 1 and n over the two with -1 <= t + n < 1, in the order
    (m0, n0), (m0, n0 + 1), (m0 + 1, n0), (m0 + 1, n0 + 1).  Returns (N, 4, 2)
    integers."""
    st = lattice_coords(e1, e2, centre, ys)
    m0 = np.ceil(-1.0 - st[:, 0]).astype(np.int64)
    n0 = np.ceil(-1.0 - st[:, 1]).astype(np.int64)
    out = [np.stack([m0 + dm, n0 + dn], axis=1) for dm in (0, 1) for dn in (0, 1)]
    return np.stack(out, axis=1)


def utilde_shifts(e1, e2, centre, ys):
    """The translates of utilde_images as vectors m e1 + n e2, (N, 4, 2)."""
    mn = utilde_images(e1, e2, centre, ys).astype(np.float64)
    return mn[..., :1] * np.asarray(e1)[None, None, :] + mn[..., 1:] * np.asarray(e2)[None, None, :]


def wrap_images(e1, e2, centre, xs):
    """Per point the integer pair (m, n) with x + m e1 + n e2 inside the unit
    cell U: lattice coordinates in [-1/2, 1/2).  Returns (N, 2) integers."""
    st = lattice_coords(e1, e2, centre, xs)
    return -np.floor(st + 0.5).astype(np.int64)


def expand_images(ys, qs, shifts_js):
    """Source list of the per-source images: positions (N K, 2), strengths,
    and for every source the index of its zero-shift copy (-1 if none)."""
    N, K, _ = shifts_js.shape
    Y = (np.asarray(ys)[:, None, :] + shifts_js).reshape(-1, 2)
    Q = np.repeat(np.asarray(qs), K, axis=0)
    zero = np.all(shifts_js == 0.0, axis=2)
    own = np.where(zero.any(axis=1), np.arange(N) * K + zero.argmax(axis=1), -1)
    return Y, Q, own


def near_discrepancy_utilde(e1, e2, centre, m, ys, qs, imgmn, mu):
    """g = [g1; g2; g3; g4] of the doubled-cell near sum (Def. Gnear) with
    the cancellation Sec. 6.2 step 2 points out.  A node y whose images have
    m in {m0, m0 + 1} (and n in {n0, n0 + 1}) contributes to
    S_near(x + e1) - S_near(x) on L, by translation invariance,
        sum_n K(x, y + (m0 - 1) e1 + n e2) - K(x, y + (m0 + 1) e1 + n e2),
    two terms per image row, each at least half a cell from L even when the
    node's body crosses a wall; likewise for U - D with the roles of e1 and
    e2 exchanged.  imgmn: per node its four (m, n) pairs (utilde_images)."""
    xl, xd, _, _ = collocation(e1, e2, centre, m)
    nl, nd = wall_normals(e1, e2)
    e1, e2 = np.asarray(e1), np.asarray(e2)
    m0 = imgmn[:, 0, 0]
    n0 = imgmn[:, 0, 1]
    nlm = np.repeat(nl[None, :], m, axis=0)
    ndm = np.repeat(nd[None, :], m, axis=0)
    zero = [np.zeros(2)]
    g = [np.zeros((m, 2)) for _ in range(4)]
    for dn in (0, 1):
        # L - R: rows n0 + dn, columns m0 - 1 (plus) and m0 + 1 (minus)
        yp = ys + (m0 - 1)[:, None] * e1[None, :] + (n0 + dn)[:, None] * e2[None, :]
        ym = ys + (m0 + 1)[:, None] * e1[None, :] + (n0 + dn)[:, None] * e2[None, :]
        g[0] += near_velocity(xl, yp, qs, zero, mu) - near_velocity(xl, ym, qs, zero, mu)
        g[1] += near_traction(xl, nlm, yp, qs, zero) - near_traction(xl, nlm, ym, qs, zero)
    for dm in (0, 1):
        # D - U: columns m0 + dm, rows n0 - 1 (plus) and n0 + 1 (minus)
        yp = ys + (m0 + dm)[:, None] * e1[None, :] + (n0 - 1)[:, None] * e2[None, :]
        ym = ys + (m0 + dm)[:, None] * e1[None, :] + (n0 + 1)[:, None] * e2[None, :]
        g[2] += near_velocity(xd, yp, qs, zero, mu) - near_velocity(xd, ym, qs, zero, mu)
        g[3] += near_traction(xd, ndm, yp, qs, zero) - near_traction(xd, ndm, ym, qs, zero)
    return np.concatenate([_split(v) for v in g])


def near_discrepancy_images(e1, e2, centre, m, Y, Q, mu):
    """g = [g1; g2; g3; g4] of a near sum given as an explicit source list
    (positions Y, strengths Q), evaluated literally as S(R) - S(L) and
    S(U) - S(D) at the collocation points (Sec. 6.2 step 2)."""
    xl, xd, _, _ = collocation(e1, e2, centre, m)
    nl, nd = wall_normals(e1, e2)
    zero = [np.zeros(2)]
    nlm = np.repeat(nl[None, :], m, axis=0)
    ndm = np.repeat(nd[None, :], m, axis=0)
    g1 = near_velocity(xl + e1, Y, Q, zero, mu) - near_velocity(xl, Y, Q, zero, mu)
    g2 = near_traction(xl + e1, nlm, Y, Q, zero) - near_traction(xl, nlm, Y, Q, zero)
    g3 = near_velocity(xd + e2, Y, Q, zero, mu) - near_velocity(xd, Y, Q, zero, mu)
    g4 = near_traction(xd + e2, ndm, Y, Q, zero) - near_traction(xd, ndm, Y, Q, zero)
    return np.concatenate([_split(g1), _split(g2), _split(g3), _split(g4)])
