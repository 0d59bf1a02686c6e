"""Write tests/golden/config2_steps.npz: three forward-Euler steps (Sec. 7) of
the 25-ellipse cell (area fraction 0.3, 256 nodes per body, dt = 1e-3) by the
FP64 oracle alone, from a zero GMRES start to a true relative residual of
1e-12 (a hundredth of the Sec. 8 tolerance, so that the stored solution's
own error stays far below the 1e-9 parity bar), with the same proxy and
collocation counts as the GPU context (M = 48 on a circle of radius 1.5,
m = 24).

Stored per step k = 0, 1, 2 (geometry at t_k = k dt): the density sigma_k
(N x 2), the rigid-body velocities v_k (n_bodies x 2) and rotation rates
omega_k (Eq. RigidBodyMotion, reading of the velocity constant as in the
oracle), mu_eff_k (particle-stress average), GMRES iterations and residual;
and the states (t, e2, x^c, theta) for k = 0..3.

Only oracle/ computes; the body descriptions come from the seeded workload
generator.  The operator is the oracle's own, evaluated at target chunks in
spawned worker processes (the same arithmetic per target as the serial
matvec).  Run from the repository root:
    python tests/golden/make_config2_step.py [--procs 8]
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import bie, geometry  # noqa: E402
from paper_1912_04501_gb300 import workloads  # noqa: E402

_OP = None


def _init(susp, kw):
    global _OP
    _OP = bie.Operator(susp, **kw)


def _rows(args):
    v, idx = args
    return _OP.apply(v.reshape(-1, 2), targets=idx)


class ParallelOperator(bie.Operator):
    """bie.Operator whose matvec evaluates chunks of targets in a pool."""
    procs = 8

    def __init__(self, susp, **kw):
        super().__init__(susp, **kw)
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_init, initargs=(susp, kw))
        self.chunks = np.array_split(np.arange(susp.N), self.procs)

    def matvec(self, v):
        v = np.asarray(v, dtype=np.float64)
        parts = self.pool.map(_rows, [(v, c) for c in self.chunks])
        return np.concatenate(parts).ravel()

    def shutdown(self):
        self.pool.close()
        self.pool.join()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=8)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "config2_steps.npz"))
    args = ap.parse_args()
    ParallelOperator.procs = args.procs
    cell = workloads.config2()
    sv = cell["solver"]
    kw = dict(n_proxy=sv["n_proxy"], proxy_radius=sv["proxy_radius"], n_coll=sv["n_coll"])
    dt = cell["dt"]
    s = geometry.Suspension(cell["e1"], cell["e2"], cell["centre"], cell["mu"], cell["gamma"], cell["bodies"])
    t = 0.0
    rec = {k: [] for k in ("t", "e2", "xc", "theta", "sigma", "v", "omega", "mu_eff", "iters", "res")}

    def state(s, t):
        rec["t"].append(t)
        rec["e2"].append(np.array(s.e2))
        rec["xc"].append(np.array([b["xc"] for b in s.bodies], dtype=np.float64))
        rec["theta"].append(np.array([b["theta"] for b in s.bodies], dtype=np.float64))

    state(s, t)
    for k in range(args.steps):
        t0 = time.time()
        ops = []

        def make(susp, **kw2):
            op = ParallelOperator(susp, **kw2)
            ops.append(op)
            return op

        s, t, out = bie.euler_step(s, cell["e2"], t, dt, kw, tol=args.tol, operator=make)
        for op in ops:
            op.shutdown()
        for key in ("sigma", "v", "omega", "mu_eff", "iters", "res"):
            rec[key].append(np.asarray(out[key]))
        state(s, t)
        print(f"step {k}: {out['iters']} iterations, residual {out['res']:.2e}, mu_eff {out['mu_eff']:.12f}, "
              f"{time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(args.out, **{k: np.array(v) for k, v in rec.items()},
                        dt=dt, seed=2, n_proxy=sv["n_proxy"], n_coll=sv["n_coll"], tol=args.tol)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
