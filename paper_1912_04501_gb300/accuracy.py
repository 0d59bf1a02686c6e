"""Per-quantity error of the mixed-precision solve against the plain FP64
solve, on the GPU, for the large cells (the 100-ellipse near-jamming cell,
the 64-cell ensemble, the 400-ellipse cell).

For each cell, from its initial geometry: the plain FP64 solve (zero start,
double-precision pair sums, GMRES to a relative residual of 1e-10) and the
default mixed solve (single-precision pairs inside iterative refinement with
double-float residuals, to the same residual) are compared on every body's
velocity and rotation rate (Sec. 3, Eq. RigidBodyMotion) and every cell's
effective viscosity (particle-stress average), as max |difference|, and on
the density as max |difference| / max |sigma|.  The FP64 solve itself is
checked against the FP64 oracle on sampled targets by the parity tests; this
measures what the mixed path adds.

Every solve runs in the library's kernels; this module only sets up the
cells and collects the results.

    python -m paper_1912_04501_gb300.accuracy [config3 config4 config5]
"""
import argparse
import json
import time

import numpy as np

from . import bie, workloads


def compare(name, gmres_max=200):
    cell = getattr(workloads, name)()
    out = {"workload": name}
    res = {}
    for label, prec in (("fp64", bie.BIE_FP64), ("mixed", bie.BIE_MIXED)):
        ctx = bie.Context(cell, precision=prec, gmres_max=gmres_max)
        t0 = time.perf_counter()
        sigma, info = ctx.solve()
        dt = time.perf_counter() - t0
        v, om, mu = ctx.velocities(sigma)
        res[label] = dict(sigma=sigma, v=v, omega=om, mu=np.atleast_1d(mu), info=info, s=dt)
        out[f"{label}_solve"] = dict(iterations=info["iterations"], rel_residual=info["rel_residual"], seconds=dt)
        out["N"] = ctx.N
        ctx.close()
    a, b = res["mixed"], res["fp64"]
    out["max_dv"] = float(np.abs(a["v"] - b["v"]).max())
    out["max_v"] = float(np.abs(b["v"]).max())
    out["max_domega"] = float(np.abs(a["omega"] - b["omega"]).max())
    out["max_dmu_eff"] = float(np.abs(a["mu"] - b["mu"]).max())
    out["sigma_rel"] = float(np.abs(a["sigma"] - b["sigma"]).max() / np.abs(b["sigma"]).max())
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cells", nargs="*", default=["config3", "config4", "config5"])
    a = ap.parse_args()
    for name in a.cells:
        print(json.dumps(compare(name)), flush=True)


if __name__ == "__main__":
    main()
