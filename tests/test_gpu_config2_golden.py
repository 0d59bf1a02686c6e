"""Solve- and step-level parity on the 25-ellipse benchmark cell (6400 nodes)
against the FP64 oracle (Sec. 3 Eq. RigidBodyMotion and Eq. mueff; Sec. 7
forward Euler).

tests/golden/config2_steps.npz holds three oracle Euler steps (dt = 1e-3,
zero GMRES start, true relative residual 1e-12), written by
tests/golden/make_config2_step.py, which calls only oracle/.  The GPU runs
the same three steps through the C ABI and every density, velocity,
rotation rate, effective viscosity and new state is compared elementwise.

* test_config2_steps_match_oracle: the plain FP64 mode and the benchmark's
  mixed mode (single-precision pairs inside FP64-class refinement,
  warm_start 2 with the shipped network: the first step starts from zero,
  the second from recycled directions, the third also from the network's
  prediction), both solved to 1e-12 like the oracle, so that each side's
  solution is within cond(A) x 1e-12 of the exact discrete solution: 1e-9
  of each quantity's scale is the bar (velocities: of max |v|; rotation
  rates: of gamma; densities: of max |sigma|; mu_eff: of mu).  Positions
  move by dt v, so their bar is dt x 1e-9 per step taken.
* test_config2_benchmark_options: exactly the benchmark's options
  (gmres_tol 1e-10).  A solution with relative residual <= 1e-10 may be off
  by cond(A) x 1e-10; on this cell the mixed solve's measured errors are
  7e-9 (sigma), 6e-10 (v), 3e-8 (omega), 1.4e-9 (mu_eff), so the stated
  mixed-mode tolerance at the benchmark's residual is 3e-8, 3e-9, 1e-7 and
  1e-8 of the same scales (a condition number of up to ~300 times the
  residual tolerance).
"""
import os

import numpy as np
import pytest

from paper_1912_04501_gb300 import workloads

pytestmark = pytest.mark.gpu

bie = pytest.importorskip("paper_1912_04501_gb300.bie")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config2_steps.npz")
TOL = 1e-9
BENCH_TOL = dict(sigma=3e-8, v=3e-9, omega=1e-7, mu_eff=1e-8)


def _unwrap(d, e1, e2, ref):
    """d minus the lattice vector that brings it closest to ref."""
    L = np.column_stack([e1, e2])
    ab = np.linalg.solve(L, (d - ref).T).T
    return d - (L @ np.round(ab).T).T


def _context(cell, mode, **kw):
    if mode == "fp64":
        return bie.Context(cell, precision=bie.BIE_FP64, warm_start=0, **kw), None
    from paper_1912_04501_gb300 import learn
    net = learn.default_net()
    ctx = bie.Context(cell, precision=bie.BIE_MIXED, warm_start=2 if net is not None else 3, **kw)
    if net is not None:
        ctx.set_warm_net(net)
    return ctx, net


def _run(ctx, g, cell, res_bar):
    """Three steps; per step the errors of sigma, v, omega, mu_eff (relative
    to their scales) and of the new positions and angles (absolute)."""
    dt = float(g["dt"])
    st = ctx.get_state()
    np.testing.assert_allclose(st["xc"], g["xc"][0], atol=1e-15)
    errs = []
    for k in range(g["sigma"].shape[0]):
        before = ctx.get_state()
        mu, info = ctx.step(dt, 1)
        assert info["rel_residual"] <= res_bar
        after = ctx.get_state()
        sig = after["sigma"].reshape(-1, 2)
        ref = g["sigma"][k]
        d = _unwrap(after["xc"] - before["xc"], np.array([1.0, 0.0]), after["e2"], dt * g["v"][k])
        v = d / dt
        om = (after["theta"] - before["theta"]) / dt
        np.testing.assert_allclose(after["e2"], g["e2"][k + 1], atol=1e-15)
        np.testing.assert_allclose(after["t"], g["t"][k + 1], atol=1e-15)
        errs.append(dict(
            sigma=np.abs(sig - ref).max() / np.abs(ref).max(),
            v=np.abs(v - g["v"][k]).max() / np.abs(g["v"][k]).max(),
            omega=np.abs(om - g["omega"][k]).max() / cell["gamma"],
            mu_eff=abs(float(mu[0]) - float(g["mu_eff"][k])) / cell["mu"],
            xc=np.abs(_unwrap(after["xc"], np.array([1.0, 0.0]), after["e2"], g["xc"][k + 1]) - g["xc"][k + 1]).max(),
            theta=np.abs(after["theta"] - g["theta"][k + 1]).max()))
    return errs


@pytest.mark.parametrize("mode", ["fp64", "mixed_learned"])
def test_config2_steps_match_oracle(mode):
    g = np.load(GOLDEN)
    assert float(g["tol"]) <= 1e-12
    cell = workloads.config2()
    assert float(g["dt"]) == cell["dt"]
    ctx, net = _context(cell, mode, gmres_tol=1e-12)
    errs = _run(ctx, g, cell, 1e-12)
    print(mode, errs)
    dt = float(g["dt"])
    for k, e in enumerate(errs):
        assert e["sigma"] < TOL and e["v"] < TOL and e["omega"] < TOL and e["mu_eff"] < TOL, (k, e)
        assert e["xc"] < (k + 1) * dt * TOL and e["theta"] < (k + 1) * dt * TOL, (k, e)
    if net is not None:
        ctx.set_warm_net(None)
        net.close()
    ctx.close()


def test_config2_benchmark_options():
    g = np.load(GOLDEN)
    cell = workloads.config2()
    ctx, net = _context(cell, "mixed_learned")
    errs = _run(ctx, g, cell, 1e-10)
    print("benchmark options", errs)
    dt = float(g["dt"])
    for k, e in enumerate(errs):
        for q, bar in BENCH_TOL.items():
            assert e[q] < bar, (k, q, e)
        assert e["xc"] < (k + 1) * dt * BENCH_TOL["v"] and e["theta"] < (k + 1) * dt * BENCH_TOL["omega"], (k, e)
    if net is not None:
        ctx.set_warm_net(None)
        net.close()
    ctx.close()
