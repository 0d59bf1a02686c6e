"""Quasi-static convergence study of Sec. 8, Example 1: two ellipses with
semi-axes (0.25, 0.125) and (0.125, 0.25) a gap d apart, solved at several
node counts N per ellipse; the linear and angular velocities are compared
with a finer reference solve.  The paper shows spectral convergence in N
with an onset that scales like 1/sqrt(d), and about 6000 nodes per ellipse
for 1e-8 accuracy at d = 1e-5 (against 1e4 nodes).

Every solve runs in the library's kernels; this module only sets up the
cells and collects the results.

    python -m paper_1912_04501_gb300.convergence [--gaps 1e-1 1e-3 1e-5]
"""
import argparse
import time

import numpy as np

from . import bie, workloads

# node counts per ellipse for each gap (the paper's ranges) and the
# reference count
STUDY = {
    1e-1: ([32, 48, 64, 96, 128], 1024),
    1e-3: ([128, 256, 384, 512, 768, 1024], 4096),
    1e-5: ([1024, 2048, 3072, 4096, 6144, 8192], 10000),
}


def solve_two_ellipses(gap, n, precision=bie.BIE_MIXED, gmres_tol=1e-10, gmres_max=1000, max_refine=12, precond=1):
    """One quasi-static solve; returns a dict with the body velocities, the
    solve statistics and the wall times of the set-up (geometry, proxy fit,
    close-evaluation blocks) and of the solve.  Near contact the system needs
    hundreds of GMRES iterations per sweep, hence long cycles (gmres_max),
    and the contact-block preconditioner (precond) cuts them several-fold.
    At d = 1e-5 the single-precision sweeps stall and the solver continues on
    the double-float operator; the residual then levels off near 1e-9, which
    is reported (allow_noconv) rather than raised."""
    import torch
    cell = workloads.two_ellipses(gap, n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = bie.Context(cell, precision=precision, gmres_tol=gmres_tol, gmres_max=gmres_max,
                      max_refine=max_refine, precond=precond)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    sigma, info = ctx.solve(allow_noconv=True)
    v, om, _ = ctx.velocities(sigma)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    npairs, under = ctx.close_info()
    ctx.close()
    return dict(gap=gap, n=n, v=v, omega=om, iterations=info["iterations"], refinements=info["refinements"],
                rel_residual=info["rel_residual"], close_pairs=npairs, under_resolved=under,
                setup_s=t1 - t0, solve_s=t2 - t1)


def study(gap, ns, n_ref, precision=bie.BIE_MIXED, precond=1, log=None):
    """Errors max|v - v_ref| and max|omega - omega_ref| over both bodies for
    each N in ns, the reference being the solve with n_ref nodes."""
    ref = solve_two_ellipses(gap, n_ref, precision, precond=precond)
    if log:
        log(f"d={gap:g} reference N={n_ref}: {ref['iterations']} its, {ref['close_pairs']} close pairs, "
            f"set-up {ref['setup_s']:.2f} s, solve {ref['solve_s']:.2f} s")
    rows = []
    for n in ns:
        r = solve_two_ellipses(gap, n, precision, precond=precond)
        r["err_v"] = float(np.abs(r["v"] - ref["v"]).max())
        r["err_omega"] = float(np.abs(r["omega"] - ref["omega"]).max())
        rows.append(r)
        if log:
            log(f"d={gap:g} N={n:6d}: err v {r['err_v']:.2e}  err omega {r['err_omega']:.2e}  "
                f"{r['iterations']} its  residual {r['rel_residual']:.1e}  {r['close_pairs']} close pairs "
                f"({r['under_resolved']} under-resolved)  set-up {r['setup_s']:.2f} s  solve {r['solve_s']:.2f} s")
    return ref, rows


def main():
    ap = argparse.ArgumentParser(description="two-ellipse convergence study (Sec. 8, Example 1)")
    ap.add_argument("--gaps", type=float, nargs="*", default=sorted(STUDY, reverse=True))
    ap.add_argument("--fp64", action="store_true", help="plain FP64 operator instead of mixed precision")
    ap.add_argument("--no-precond", action="store_true", help="without the contact-block preconditioner")
    a = ap.parse_args()
    prec = bie.BIE_FP64 if a.fp64 else bie.BIE_MIXED
    for gap in a.gaps:
        ns, n_ref = STUDY[min(STUDY, key=lambda g: abs(np.log(g / gap)))]
        study(gap, ns, n_ref, prec, precond=0 if a.no_precond else 1, log=print)


if __name__ == "__main__":
    main()
