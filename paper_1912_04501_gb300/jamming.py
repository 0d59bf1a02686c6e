"""Star-shaped jamming runs of Sec. 8 Examples 4-5.

Two star-shaped bodies in the unit square are sheared (mu = gamma = 1,
forward Euler, dt = 5e-4, 2500 nodes per body) until they jam: mu_eff(t)
grows without bound as the gaps close.  Lubrication theory (remark after
Example 4, Eq. blowup) predicts mu_eff ~ c |t - t*|^-beta with beta = 5/2 for
a reservoir trapped between two contacts (Example 4) and 3/2 for a single
contact (Example 5); the paper fits (c, t*, beta) by nonlinear least squares
on t in [0.4, 0.44] and [0.4, 0.45].

Every solve and step runs in the library's kernels (single-precision pairs
inside FP64-class refinement, the contact-block preconditioner, long GMRES
cycles); this module sets up the cells, records mu_eff(t) and fits the power
law on the host.

    python -m paper_1912_04501_gb300.jamming [--example 4 5] [--n 2500] [--out DIR]
"""
import argparse
import json
import math
import os
import time

import numpy as np

from . import bie, workloads


TOLERANCES = (1e-10, 1e-9, 1e-8)


MIN_GAP = 1e-6  # a smaller gap between the bodies ends the run (BIE_ECOLLIDE): they touch


def _context(cell, tol, close_rule=0):
    return bie.Context(cell, precision=bie.BIE_MIXED, gmres_max=1000, max_refine=40, precond=1, gmres_tol=tol,
                       min_gap=MIN_GAP, close_rule=close_rule)


def run(example=4, n=2500, dt=5e-4, t_end=0.5, mu_stop=1e5, log=print, close_rule=0):
    """Time steps until t_end, a mu_eff above mu_stop, bodies closer than
    MIN_GAP, or a step the solver cannot finish; returns the record.  Steps solve to a relative residual
    of 1e-10; when the gaps get so small that a solve stops above it (the
    double-float residual of the near-contact terms, a few 1e-10 of the
    right-hand side), the run continues from the same state at the next
    looser tolerance of TOLERANCES, and the record notes where."""
    cell = workloads.stars(example, n)
    tol_k = 0
    ctx = _context(cell, TOLERANCES[tol_k], close_rule)
    rec = dict(example=example, n=n, dt=dt, t=[], mu_eff=[], iterations=[], residual=[], close_pairs=[],
               seconds=[], tolerance=[], stop="t_end")
    t = 0.0
    k = 0
    while t < t_end - 0.5 * dt:
        t0 = time.perf_counter()
        try:
            mu, info = ctx.step(dt, 1)
        except bie.BieError as e:
            if e.code == bie.BIE_ENOCONV and tol_k + 1 < len(TOLERANCES):
                st = ctx.get_state()
                ctx.close()
                tol_k += 1
                ctx = _context(cell, TOLERANCES[tol_k], close_rule)
                ctx.set_state(st["t"], st["e2"], st["xc"], st["theta"], st["sigma"], st["sigma_prev2"],
                              st["dt_prev"], st["d2"])
                if log:
                    log(f"example {example}: t = {t:.4f}, tolerance now {TOLERANCES[tol_k]:g} ({e})")
                continue
            rec["stop"] = str(e)
            break
        rec["seconds"].append(time.perf_counter() - t0)
        rec["t"].append(t)  # mu_eff of the solve at time t (before the bodies move)
        rec["mu_eff"].append(float(mu[0]))
        rec["iterations"].append(info["iterations"])
        rec["residual"].append(info["rel_residual"])
        rec["close_pairs"].append(ctx.close_info()[0])
        rec["tolerance"].append(TOLERANCES[tol_k])
        t += dt
        k += 1
        if log and k % 50 == 0:
            log(f"example {example}: t = {t:.4f}, mu_eff = {mu[0]:.6g}, {info['iterations']} iterations, "
                f"{rec['close_pairs'][-1]} close pairs, {rec['seconds'][-1] * 1e3:.0f} ms")
        if float(mu[0]) > mu_stop:
            rec["stop"] = f"mu_eff above {mu_stop:g}"
            break
    ctx.close()
    return rec


def _advance(ctx, make, dt, t, t_end, tol_k, rec=None, log=None, tag=""):
    """Step ctx from t to t_end, falling back to looser TOLERANCES when a
    solve stops above its tolerance (make(tol) builds a fresh context);
    returns (ctx, t, tol_k, stop) and appends (t, mu_eff) to rec."""
    while t < t_end - 0.5 * dt:
        try:
            mu, _ = ctx.step(dt, 1)
        except bie.BieError as e:
            if e.code == bie.BIE_ENOCONV and tol_k + 1 < len(TOLERANCES):
                st = ctx.get_state()
                ctx.close()
                tol_k += 1
                ctx = make(TOLERANCES[tol_k])
                ctx.set_state(st["t"], st["e2"], st["xc"], st["theta"], st["sigma"], st["sigma_prev2"],
                              st["dt_prev"], st["d2"])
                continue
            return ctx, t, tol_k, str(e)
        if rec is not None:
            rec.append((t, float(mu[0])))
            if log:
                log(f"{tag} t = {t:.5f} mu_eff = {mu[0]:.6g} (tolerance {TOLERANCES[tol_k]:g})")
        t += dt
    return ctx, t, tol_k, "t_end"


def convergence_check(example=5, n=2500, dt=5e-4, t0=0.39, t1=0.405, log=print):
    """mu_eff(t) on [t0, t1] from the state the run reaches at t0, four ways:
    as run (mixed precision), with plain FP64 solves, with 1.6 n nodes per
    body (the bodies' positions and orientations carried over), and with
    dt / 2.  Returns {variant: [(t, mu_eff), ...], "stop": {...}}."""
    cell = workloads.stars(example, n)
    ctx = _context(cell, TOLERANCES[0])
    ctx, t, tol_k, stop = _advance(ctx, lambda tol: _context(cell, tol), dt, 0.0, t0, 0)
    st = ctx.get_state()
    ctx.close()
    out = {"stop": {}}
    n2 = int(round(1.6 * n / 8)) * 8
    variants = (("mixed", cell, bie.BIE_MIXED, dt, True), ("fp64", cell, bie.BIE_FP64, dt, True),
                (f"n{n2}", workloads.stars(example, n2), bie.BIE_MIXED, dt, False),
                ("dt/2", cell, bie.BIE_MIXED, dt / 2, True))
    for tag, c, prec, h, history in variants:
        def make(tol, c=c, prec=prec):
            return bie.Context(c, precision=prec, gmres_max=1000, max_refine=40, precond=1, gmres_tol=tol,
                               min_gap=MIN_GAP)
        ctx = make(TOLERANCES[tol_k])
        if history:
            ctx.set_state(st["t"], st["e2"], st["xc"], st["theta"], st["sigma"], st["sigma_prev2"],
                          st["dt_prev"], st["d2"])
        else:
            ctx.set_state(st["t"], st["e2"], st["xc"], st["theta"])
        rec = []
        ctx, _, _, stop = _advance(ctx, make, h, st["t"], t1, tol_k, rec, log, tag)
        ctx.close()
        out[tag] = rec
        out["stop"][tag] = stop
    return out


def fit_blowup(t, mu, window):
    """Nonlinear least squares for mu ~ c |t - t*|^-beta (Eq. blowup) on
    window = (t0, t1): the residual is taken in log mu; returns c, t*, beta
    and the relative residual of mu."""
    from scipy.optimize import least_squares
    t = np.asarray(t, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    sel = (t >= window[0]) & (t <= window[1]) & (mu > 0)
    ts, ms = t[sel], mu[sel]
    if ts.size < 5:
        raise ValueError("too few points in the fitting window")

    def res(p):
        logc, ts_, beta = p
        return logc - beta * np.log(np.maximum(ts_ - ts, 1e-12)) - np.log(ms)

    best = None
    for tstar0 in ts[-1] + np.array([1e-3, 5e-3, 2e-2, 5e-2]):
        p0 = [math.log(ms[-1]) + 2.0 * math.log(tstar0 - ts[-1]), tstar0, 2.0]
        r = least_squares(res, p0, bounds=([-50, ts[-1] + 1e-9, 0.0], [50, ts[-1] + 1.0, 10.0]))
        if best is None or r.cost < best.cost:
            best = r
    logc, tstar, beta = best.x
    fitted = math.exp(logc) * (tstar - ts) ** (-beta)
    rel = float(np.linalg.norm(fitted - ms) / np.linalg.norm(ms))
    return dict(c=math.exp(logc), t_star=float(tstar), beta=float(beta), rel_residual=rel, points=int(ts.size))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--example", type=int, nargs="*", default=[4, 5])
    ap.add_argument("--n", type=int, default=2500)
    ap.add_argument("--t-end", type=float, default=0.5)
    ap.add_argument("--out", default=None, help="directory for the mu_eff(t) records (JSON)")
    ap.add_argument("--close-rule", type=int, choices=(0, 1), default=0,
                    help="close-evaluation blocks: 0 fine trapezoidal rule, 1 the paper's barycentric rule")
    ap.add_argument("--check", nargs=2, type=float, default=None, metavar=("T0", "T1"),
                    help="instead of the runs: mu_eff on [T0, T1] as run, with FP64 solves, 1.6x the nodes "
                         "and half the step, all from the state at T0")
    a = ap.parse_args()
    if a.check:
        for ex in a.example:
            res = convergence_check(ex, a.n, t0=a.check[0], t1=a.check[1], log=None)
            print(json.dumps({"example": ex, **res}), flush=True)
            if a.out:
                os.makedirs(a.out, exist_ok=True)
                with open(os.path.join(a.out, f"jamming_check{ex}.json"), "w") as f:
                    json.dump(res, f)
        return
    for ex in a.example:
        rec = run(ex, a.n, t_end=a.t_end, close_rule=a.close_rule)
        out = dict(example=ex, n=a.n, steps=len(rec["t"]), stop=rec["stop"],
                   t_last=rec["t"][-1] if rec["t"] else None, mu_last=rec["mu_eff"][-1] if rec["mu_eff"] else None,
                   seconds=float(np.sum(rec["seconds"])),
                   tolerance_switches=[(rec["t"][k], rec["tolerance"][k]) for k in range(1, len(rec["t"]))
                                       if rec["tolerance"][k] != rec["tolerance"][k - 1]])
        out["fit"] = {}
        # the paper's window (t in [0.4, 0.44] or [0.4, 0.45]) if the run got
        # there, and the last 0.04 shear times before the run ended, where
        # mu_eff is in its asymptotic regime
        wins = {"paper": (0.40, 0.44 if ex == 4 else 0.45)}
        if rec["t"]:
            wins["last 0.04"] = (rec["t"][-1] - 0.04, rec["t"][-1])
        for name, w in wins.items():
            try:
                out["fit"][name] = dict(window=w, **fit_blowup(rec["t"], rec["mu_eff"], w))
            except (ValueError, ImportError) as e:
                out["fit"][name] = str(e)
        print(json.dumps(out), flush=True)
        if a.out:
            os.makedirs(a.out, exist_ok=True)
            with open(os.path.join(a.out, f"jamming_example{ex}.json"), "w") as f:
                json.dump(rec, f)


if __name__ == "__main__":
    main()
