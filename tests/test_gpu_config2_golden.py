"""Solve- and step-level parity on the 25-ellipse benchmark cell (6400 nodes)
against the FP64 oracle (Sec. 3 Eq. RigidBodyMotion and Eq. mueff; Sec. 7
forward Euler).

tests/golden/config2_steps.npz holds three oracle Euler steps (dt = 1e-3,
zero GMRES start, true relative residual 1e-10), written by
tests/golden/make_config2_step.py, which calls only oracle/.  The GPU runs
the same three steps through the C ABI in the plain FP64 mode and in the
benchmark's mode (single-precision pairs inside FP64-class refinement,
warm_start 2 with the shipped network: the first step starts from zero, the
second from recycled directions, the third also from the network's
prediction), and every density, velocity, rotation rate, effective
viscosity and new state is compared elementwise.

Tolerances: both sides solve to a relative residual of 1e-10 (the oracle:
||b - A sigma|| <= 1e-10 ||b||; the GPU: the same with an FP64-class
residual), so each solution carries an error of up to cond(A) x 1e-10
relative to its scale; the operator is well conditioned here (GMRES
converges in ~70 iterations), and 1e-9 of each quantity's scale is the
bar (velocities: of max |v|; rotation rates: of gamma; densities: of
max |sigma|; mu_eff: of mu).  Positions move by dt v, so their bar is
dt x 1e-9 per step taken.
"""
import os

import numpy as np
import pytest

from paper_1912_04501_gb300 import workloads

pytestmark = pytest.mark.gpu

bie = pytest.importorskip("paper_1912_04501_gb300.bie")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config2_steps.npz")
TOL = 1e-9


def _unwrap(d, e1, e2, ref):
    """d minus the lattice vector that brings it closest to ref."""
    L = np.column_stack([e1, e2])
    ab = np.linalg.solve(L, (d - ref).T).T
    return d - (L @ np.round(ab).T).T


@pytest.mark.parametrize("mode", ["fp64", "mixed_learned"])
def test_config2_steps_match_oracle(mode):
    g = np.load(GOLDEN)
    cell = workloads.config2()
    dt = float(g["dt"])
    assert dt == cell["dt"]
    if mode == "fp64":
        ctx = bie.Context(cell, precision=bie.BIE_FP64, warm_start=0)
        net = None
    else:
        from paper_1912_04501_gb300 import learn
        net = learn.default_net()
        ctx = bie.Context(cell, precision=bie.BIE_MIXED, warm_start=2 if net is not None else 3)
        if net is not None:
            ctx.set_warm_net(net)
    st = ctx.get_state()
    np.testing.assert_allclose(st["xc"], g["xc"][0], atol=1e-15)
    errs = {}
    for k in range(g["sigma"].shape[0]):
        before = ctx.get_state()
        mu, info = ctx.step(dt, 1)
        assert info["rel_residual"] <= 1e-10
        after = ctx.get_state()
        # density of the solve at t_k
        sig = after["sigma"].reshape(-1, 2)
        ref = g["sigma"][k]
        e_sig = np.abs(sig - ref).max() / np.abs(ref).max()
        # velocities and rotation rates at t_k from the Euler update
        d = _unwrap(after["xc"] - before["xc"], np.array([1.0, 0.0]), after["e2"], dt * g["v"][k])
        v = d / dt
        om = (after["theta"] - before["theta"]) / dt
        e_v = np.abs(v - g["v"][k]).max() / np.abs(g["v"][k]).max()
        e_om = np.abs(om - g["omega"][k]).max() / cell["gamma"]
        e_mu = abs(float(mu[0]) - float(g["mu_eff"][k])) / cell["mu"]
        # the new state t_{k+1}
        np.testing.assert_allclose(after["e2"], g["e2"][k + 1], atol=1e-15)
        np.testing.assert_allclose(after["t"], g["t"][k + 1], atol=1e-15)
        e_x = np.abs(_unwrap(after["xc"], np.array([1.0, 0.0]), after["e2"], g["xc"][k + 1]) - g["xc"][k + 1]).max()
        e_th = np.abs(after["theta"] - g["theta"][k + 1]).max()
        errs[k] = dict(sigma=e_sig, v=e_v, omega=e_om, mu_eff=e_mu, xc=e_x, theta=e_th)
        assert e_sig < TOL and e_v < TOL and e_om < TOL and e_mu < TOL, (k, errs[k])
        assert e_x < (k + 1) * dt * TOL and e_th < (k + 1) * dt * TOL, (k, errs[k])
    print(mode, errs)
    if net is not None:
        ctx.set_warm_net(None)
        net.close()
    ctx.close()
