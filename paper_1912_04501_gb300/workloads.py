"""Seeded synthetic suspensions (input generators only).

This module draws body descriptions -- ellipse semi-axes, centres, angles and
node counts -- for unit cells shaped like the suspensions studied in
arXiv 1912.04501 (ellipses at a given area fraction and minimum gap).  It holds
none of the boundary-integral arithmetic: it is read both by the GPU library's
callers and by the CPU oracle's tests, and imports neither.

Every function returns a plain dict:
    e1, e2, centre : lattice vectors and cell centre (lists of 2 floats)
    mu, gamma      : viscosity and shear rate
    bodies         : list of {"a", "b", "xc": [x, y], "theta", "n"}
    solver         : suggested n_proxy, proxy_radius, n_coll, gmres_tol
    dt, steps      : time-stepping parameters of the workload
"""
import math

import numpy as np

SAMPLES = 1024  # boundary samples per ellipse used by the gap estimate
FAST_SAMPLES = 256  # coarser outlines for placement loops (distance error ~1e-6 here)


def _outline(a, b, xc, theta, k=SAMPLES):
    t = 2.0 * np.pi * np.arange(k) / k
    c, s = math.cos(theta), math.sin(theta)
    px, py = a * np.cos(t), b * np.sin(t)
    return np.stack([xc[0] + c * px - s * py, xc[1] + s * px + c * py], axis=1)


def _inside(a, b, xc, theta, pts):
    c, s = math.cos(theta), math.sin(theta)
    d = pts - np.asarray(xc)[None, :]
    u = c * d[:, 0] + s * d[:, 1]
    v = -s * d[:, 0] + c * d[:, 1]
    return (u / a) ** 2 + (v / b) ** 2 < 1.0


def gap_estimate(b1, b2, shift=(0.0, 0.0), k=SAMPLES):
    """Minimum distance between two ellipse outlines sampled at k points
    each (negative if they overlap).  shift translates the second body."""
    p = _outline(b1["a"], b1["b"], b1["xc"], b1["theta"], k)
    xc2 = [b2["xc"][0] + shift[0], b2["xc"][1] + shift[1]]
    q = _outline(b2["a"], b2["b"], xc2, b2["theta"], k)
    if _inside(b1["a"], b1["b"], b1["xc"], b1["theta"], q).any() or \
            _inside(b2["a"], b2["b"], xc2, b2["theta"], p).any():
        return -1.0
    d2 = ((p[:, None, :] - q[None, :, :]) ** 2).sum(-1)
    return float(np.sqrt(d2.min()))


def min_gap(cell):
    """Smallest gap between any two bodies of the cell, periodic images
    included (sampling estimate)."""
    e1, e2 = np.asarray(cell["e1"]), np.asarray(cell["e2"])
    bodies = cell["bodies"]
    best = np.inf
    for i in range(len(bodies)):
        for j in range(i, len(bodies)):
            for m in (-1, 0, 1):
                for n in (-1, 0, 1):
                    if i == j and m == 0 and n == 0:
                        continue
                    sh = m * e1 + n * e2
                    ci, cj = np.asarray(bodies[i]["xc"]), np.asarray(bodies[j]["xc"]) + sh
                    reach = max(bodies[i]["a"], bodies[i]["b"]) + max(bodies[j]["a"], bodies[j]["b"])
                    if np.hypot(*(ci - cj)) - reach > best:
                        continue
                    best = min(best, gap_estimate(bodies[i], bodies[j], sh))
    return best


def config1():
    """Unit cell (1,0),(0,1) centred at (0.5,0.5); mu = gamma = 1; one
    ellipse 0.2 x 0.1 at the centre, angle 0, 128 nodes; 16 proxy Stokeslets
    on a circle of radius 1.5; GMRES tolerance 1e-10; 10 Euler steps of 0.01."""
    return dict(e1=[1.0, 0.0], e2=[0.0, 1.0], centre=[0.5, 0.5], mu=1.0, gamma=1.0,
                bodies=[dict(a=0.2, b=0.1, xc=[0.5, 0.5], theta=0.0, n=128)],
                solver=dict(n_proxy=16, proxy_radius=1.5, n_coll=16, gmres_tol=1e-10),
                dt=0.01, steps=10)


def random_cell(n_bodies, phi, aspect, min_gap_target, nodes, seed,
                e1=(1.0, 0.0), e2=(0.0, 1.0), centre=(0.5, 0.5), equal_area=True,
                max_tries=200000):
    """Random sequential placement of n_bodies ellipses of total area fraction
    phi and aspect ratios uniform in `aspect`, angles uniform in [0, pi), every
    gap (periodic images included) at least min_gap_target.  nodes is an int
    or a callable(a, b) -> int."""
    rng = np.random.default_rng(seed)
    e1, e2, centre = np.asarray(e1, float), np.asarray(e2, float), np.asarray(centre, float)
    area_cell = abs(e1[0] * e2[1] - e1[1] * e2[0])
    if equal_area:
        areas = np.full(n_bodies, phi * area_cell / n_bodies)
    else:
        w = rng.uniform(0.5, 1.5, n_bodies)
        areas = phi * area_cell * w / w.sum()
    bodies = []
    tries = 0
    shifts = np.array([m * e1 + n * e2 for m in (-1, 0, 1) for n in (-1, 0, 1)])
    for k in range(n_bodies):
        alpha = rng.uniform(*aspect)
        a = math.sqrt(areas[k] * alpha / math.pi)
        b = math.sqrt(areas[k] / (alpha * math.pi))
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("placement failed; lower phi or min_gap")
            uv = rng.uniform(-0.5, 0.5, 2)
            xc = centre + uv[0] * e1 + uv[1] * e2
            cand = dict(a=a, b=b, xc=[float(xc[0]), float(xc[1])], theta=float(rng.uniform(0, math.pi)))
            ok = True
            if bodies:
                cen = np.array([o["xc"] for o in bodies])
                rad = np.array([max(o["a"], o["b"]) for o in bodies])
                d = np.linalg.norm(cen[:, None, :] + shifts[None, :, :] - xc[None, None, :], axis=2)
                near = np.argwhere(d - (max(a, b) + rad[:, None]) <= min_gap_target)
                for j, s_ in near:
                    if gap_estimate(cand, bodies[j], shifts[s_], FAST_SAMPLES) < min_gap_target:
                        ok = False
                        break
            if ok:
                break
        cand["n"] = int(nodes(a, b) if callable(nodes) else nodes)
        bodies.append(cand)
    return dict(e1=e1.tolist(), e2=e2.tolist(), centre=centre.tolist(), mu=1.0, gamma=1.0,
                bodies=bodies)


def config2(seed=2):
    """25 equal-area ellipses, area fraction 0.3, aspect ratios uniform in
    [1, 3], minimum gap 1e-2, 256 nodes per body (6400 nodes); 100 Euler
    steps of 1e-3 with the lattice skewing."""
    cell = random_cell(25, 0.3, (1.0, 3.0), 1e-2, 256, seed)
    cell.update(solver=dict(n_proxy=48, proxy_radius=1.5, n_coll=24, gmres_tol=1e-10),
                dt=1e-3, steps=100)
    return cell


def small_cell(n_bodies=3, nodes=64, seed=0, phi=0.2, gap=0.05, e2=(0.0, 1.0)):
    """A few-body cell for quick parity checks (several tiles, ragged sizes)."""
    cell = random_cell(n_bodies, phi, (1.0, 2.5), gap,
                       nodes if callable(nodes) else (lambda a, b, _n=nodes: _n), seed, e2=e2,
                       equal_area=False)
    cell.update(solver=dict(n_proxy=32, proxy_radius=1.5, n_coll=16, gmres_tol=1e-10),
                dt=1e-3, steps=2)
    return cell


def two_ellipses(gap, n, mu=1.0, gamma=1.0):
    """The two ellipses of the paper's quasi-static convergence example
    (Sec. 8, Example 1): semi-axes (0.25, 0.125) and (0.125, 0.25), centres on
    a horizontal line with |x1 - x2| = gap + 0.375, here placed in the unit
    cell (1,0),(0,1) centred at (0.5, 0.5) (the paper does not give the cell,
    mu or gamma)."""
    half = 0.5 * (gap + 0.375)
    return dict(e1=[1.0, 0.0], e2=[0.0, 1.0], centre=[0.5, 0.5], mu=mu, gamma=gamma,
                bodies=[dict(a=0.25, b=0.125, xc=[0.5 - half, 0.5], theta=0.0, n=n),
                        dict(a=0.125, b=0.25, xc=[0.5 + half, 0.5], theta=0.0, n=n)],
                solver=dict(n_proxy=48, proxy_radius=1.5, n_coll=24, gmres_tol=1e-10),
                dt=1e-3, steps=1)


def _neighbour_gaps(bodies, e1, e2, i, reach_pad, k=FAST_SAMPLES):
    """Gaps of body i to every other body (and its own images) within reach."""
    bi = bodies[i]
    shifts = np.array([m * e1 + n * e2 for m in (-1, 0, 1) for n in (-1, 0, 1)])
    cen = np.array([o["xc"] for o in bodies])
    rad = np.array([max(o["a"], o["b"]) for o in bodies])
    d = np.linalg.norm(cen[:, None, :] + shifts[None, :, :] - np.asarray(bi["xc"])[None, None, :], axis=2)
    near = np.argwhere(d - (max(bi["a"], bi["b"]) + rad[:, None]) <= reach_pad)
    out = []
    for j, s_ in near:
        if j == i and s_ == 4:
            continue
        out.append(gap_estimate(bi, bodies[j], shifts[s_], k))
    return out


def compress(cell, phi_target, min_gap_target, seed, step=0.01, moves=30, max_rounds=400):
    """Raise the area fraction of a placed cell to phi_target: alternate a
    uniform inflation of every body's size and Monte-Carlo displacements
    (random small moves and rotations, rejected if any gap falls below
    min_gap_target).  Deterministic for a given seed."""
    rng = np.random.default_rng(seed)
    e1, e2 = np.asarray(cell["e1"], float), np.asarray(cell["e2"], float)
    area_cell = abs(e1[0] * e2[1] - e1[1] * e2[0])
    bodies = [dict(b) for b in cell["bodies"]]
    phi = lambda: sum(math.pi * b["a"] * b["b"] for b in bodies) / area_cell
    for _ in range(max_rounds):
        if phi() >= phi_target - 1e-12:
            break
        f = min(1.0 + step, math.sqrt(phi_target / phi()))
        trial = [dict(b, a=b["a"] * f, b=b["b"] * f) for b in bodies]
        bad = [i for i in range(len(trial)) if min(_neighbour_gaps(trial, e1, e2, i, 0.05) or [1.0]) < min_gap_target]
        # relieve the offending bodies by random moves at the inflated size
        for i in bad:
            for _ in range(moves):
                old = trial[i]
                cand = dict(old, xc=[old["xc"][0] + rng.normal(0, 0.01), old["xc"][1] + rng.normal(0, 0.01)],
                            theta=old["theta"] + rng.normal(0, 0.05))
                trial[i] = cand
                if min(_neighbour_gaps(trial, e1, e2, i, 0.05) or [1.0]) >= min_gap_target:
                    break
                trial[i] = old
        if all(min(_neighbour_gaps(trial, e1, e2, i, 0.05) or [1.0]) >= min_gap_target for i in bad):
            bodies = trial
        else:
            step *= 0.5
            if step < 1e-4:
                break
        # a sweep of random moves everywhere keeps the packing from locking up
        for i in rng.permutation(len(bodies))[: len(bodies) // 4]:
            old = bodies[i]
            bodies[i] = dict(old, xc=[old["xc"][0] + rng.normal(0, 0.005), old["xc"][1] + rng.normal(0, 0.005)])
            if min(_neighbour_gaps(bodies, e1, e2, i, 0.05) or [1.0]) < min_gap_target:
                bodies[i] = old
    out = dict(cell)
    out["bodies"] = bodies
    return out


def config3(seed=3):
    """Near jamming: 100 ellipses, aspect ratios uniform in [1, 2], placed at
    area fraction 0.30 and compressed to 0.45 with every gap >= 1e-3; nodes
    per body N_i = clamp(8 ceil(C P_i / (8 sqrt(d_i))), 128, 512), d_i the
    body's smallest gap, C such that a gap of 1e-3 gets 512 nodes at the mean
    perimeter."""
    cell = random_cell(100, 0.30, (1.0, 2.0), 1e-2, 128, seed, equal_area=False)
    cell = compress(cell, 0.45, 1e-3, seed)
    e1, e2 = np.asarray(cell["e1"], float), np.asarray(cell["e2"], float)
    bodies = cell["bodies"]
    per = [math.pi * (3 * (b["a"] + b["b"]) - math.sqrt((3 * b["a"] + b["b"]) * (b["a"] + 3 * b["b"])))
           for b in bodies]
    cconst = 512.0 * math.sqrt(1e-3) / np.mean(per)
    for i, b in enumerate(bodies):
        d = max(min(_neighbour_gaps(bodies, e1, e2, i, 0.2) or [0.1]), 1e-4)
        b["n"] = int(min(512, max(128, 8 * math.ceil(cconst * per[i] / (8 * math.sqrt(d))))))
    cell.update(solver=dict(n_proxy=48, proxy_radius=1.5, n_coll=24, gmres_tol=1e-10), dt=1e-3, steps=10)
    return cell


def config4(seed=4, n_cells=64):
    """Batched ensemble: n_cells independent unit cells, cell c drawn with
    seed seed + c: body count uniform in {5..50}, area fraction uniform in
    [0.1, 0.4], aspect ratios uniform in [1, 3], minimum gap 1e-2, nodes per
    body clamp(8 ceil(P_i / (8 h*)), 128, 256) with h* = the mean perimeter
    over 160 (so a typical body gets ~160 nodes)."""
    cells = []
    for c in range(n_cells):
        rng = np.random.default_rng(seed + c)
        nb = int(rng.integers(5, 51))
        phi = float(rng.uniform(0.1, 0.4))
        cell = random_cell(nb, phi, (1.0, 3.0), 1e-2, 128, seed + c)
        per = [math.pi * (3 * (b["a"] + b["b"]) - math.sqrt((3 * b["a"] + b["b"]) * (b["a"] + 3 * b["b"])))
               for b in cell["bodies"]]
        hstar = np.mean(per) / 160.0
        for b, p_ in zip(cell["bodies"], per):
            b["n"] = int(min(256, max(128, 8 * math.ceil(p_ / (8 * hstar)))))
        cell.update(solver=dict(n_proxy=48, proxy_radius=1.5, n_coll=24, gmres_tol=1e-10), dt=1e-3, steps=10)
        cells.append(cell)
    return cells


def config5(seed=5):
    """400 ellipses, area fraction 0.35, aspect ratios uniform in [1, 3],
    minimum gap 2e-3, 256 nodes per body (102400 nodes); 50 Euler steps of
    1e-3.  (A gap of 1e-2 would be a third of the smaller semi-axes at this
    size -- an effective area fraction near 0.6 that random placement and
    compression do not reach.)"""
    cell = random_cell(400, 0.35, (1.0, 3.0), 2e-3, 256, seed, max_tries=2000000)
    cell.update(solver=dict(n_proxy=48, proxy_radius=1.5, n_coll=24, gmres_tol=1e-10), dt=1e-3, steps=50)
    return cell


# Arms of the star shapes of Sec. 8 Examples 4-5.  The printed radius
# r = 0.25 (1 + 0.5 cos theta) has a single lobe (the multiplier of theta is
# lost in the text); four arms keep both examples' initial stars apart
# (three, five and six arms overlap the second example's rotated star).
STAR_ARMS = 4


def stars(example=4, n=2500, arms=STAR_ARMS):
    """Two star-shaped bodies r(t) = r0 (1 + 0.5 cos(arms t)) in the unit
    square cell, centred at (0.25, 0.25) and (0.75, 0.75), mu = gamma = 1,
    forward Euler with dt = 5e-4 (Sec. 8 Example 4: r0 = 0.25; Example 5:
    r0 = 0.275 and the second star turned by pi/4), n nodes per body."""
    r0 = 0.25 if example == 4 else 0.275
    th2 = 0.0 if example == 4 else np.pi / 4
    bodies = [dict(shape="star", r0=r0, eps=0.5, k=arms, xc=[0.25, 0.25], theta=0.0, n=n),
              dict(shape="star", r0=r0, eps=0.5, k=arms, xc=[0.75, 0.75], theta=th2, n=n)]
    return dict(e1=[1.0, 0.0], e2=[0.0, 1.0], centre=[0.5, 0.5], mu=1.0, gamma=1.0, bodies=bodies,
                solver=dict(n_proxy=64, proxy_radius=1.5, n_coll=32, gmres_tol=1e-10), dt=5e-4, steps=920)
