"""GPU tests at near contact (Sec. 8, Example 1 at d = 1e-5): the close-
evaluation blocks with fine rules up to 1024-fold upsampling and bodies of
more nodes than one block-building CTA holds, against the oracle's
definition of the correction on the targets nearest the contact.

Tolerances as in the other parity tests: FP64 and double-float 1e-10,
single-precision pairs 5e-5 (relative to the largest sampled entry).
"""
import numpy as np
import pytest

from paper_1912_04501_gb300 import workloads
from tests.conftest import oracle_operator

pytestmark = pytest.mark.gpu

bie = pytest.importorskip("paper_1912_04501_gb300.bie")


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("gap,n", [(1e-5, 512), (1e-5, 6144)])
def test_close_parity_at_gap_1e5(gap, n):
    """n = 512: the closest targets need the 1024-fold rule (tables beyond
    the 64-fold ones built at start-up); n = 6144: 128-fold, and each block
    is built by two CTAs (node ranges of 4096)."""
    cell = workloads.two_ellipses(gap, n)
    ctx = bie.Context(cell, precision=bie.BIE_FP64)
    npairs, under = ctx.close_info()
    assert npairs > 0 and under == 0
    x, _, _, _ = ctx.nodes()
    # targets nearest the contact point on each body, and a few others
    contact = np.array([0.5625, 0.5])  # the tips face each other there
    dist = np.linalg.norm(x - contact[None, :], axis=1)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([np.argsort(dist[:n])[:6], n + np.argsort(dist[n:])[:6],
                                    rng.choice(2 * n, 4, replace=False)]))
    op = oracle_operator(cell, close_targets=idx)
    sigma = rng.standard_normal(2 * ctx.N)
    ref = op.apply(sigma.reshape(-1, 2), targets=idx)
    for prec, tol in ((bie.BIE_FP64, 1e-10), (bie.BIE_DF64, 1e-10), (bie.BIE_MIXED, 5e-5)):
        y = ctx.apply(sigma, precision=prec).reshape(-1, 2)[idx]
        assert _rel(y, ref) < tol, (prec, _rel(y, ref))
    ctx.close()


@pytest.mark.parametrize("gap", [2e-3, 1e-5])
def test_close_evaluation_matches_the_papers_rule(gap):
    """The GPU's close-evaluation blocks (the fine rule of the interpolated
    density) against the oracle evaluating the same pairs by the paper's own
    special quadrature (Sec. 6.3: compensated barycentric Cauchy integrals,
    oracle/barycentric.py), on a smooth density, at the targets nearest the
    contact: FP64 and double-float to 1e-10."""
    n = 512
    cell = workloads.two_ellipses(gap, n)
    ctx = bie.Context(cell, precision=bie.BIE_FP64)
    x, _, _, _ = ctx.nodes()
    contact = np.array([0.5625, 0.5])
    dist = np.linalg.norm(x - contact[None, :], axis=1)
    idx = np.unique(np.concatenate([np.argsort(dist[:n])[:8], n + np.argsort(dist[n:])[:8]]))
    op = oracle_operator(cell, close_targets=idx, close_rule="barycentric")
    assert len(op.close.pairs) >= 16
    sigma = []
    for k, b in enumerate(cell["bodies"]):
        t = 2 * np.pi * np.arange(b["n"]) / b["n"]
        sigma.append(np.stack([np.cos(2 * t + k) + 0.3 * np.sin(5 * t), 0.5 * np.sin(3 * t - k) + 0.2], axis=1))
    sigma = np.concatenate(sigma)
    ref = op.apply(sigma, targets=idx)
    for prec in (bie.BIE_FP64, bie.BIE_DF64):
        y = ctx.apply(sigma.ravel(), precision=prec).reshape(-1, 2)[idx]
        assert _rel(y, ref) < 1e-10, (prec, _rel(y, ref))
    ctx.close()


@pytest.mark.parametrize("gap,n", [(2e-3, 256), (1e-5, 512)])
def test_barycentric_blocks_match_the_oracle(gap, n):
    """opts.close_rule = 1 builds the blocks by the paper's rule on the GPU:
    against the oracle's barycentric rule (the same quadrature) on a random
    density, FP64 and double-float to 1e-10, single-precision pairs 5e-5."""
    cell = workloads.two_ellipses(gap, n)
    ctx = bie.Context(cell, precision=bie.BIE_FP64, close_rule=1)
    npairs, under = ctx.close_info()
    assert npairs > 0 and under == 0
    x, _, _, _ = ctx.nodes()
    contact = np.array([0.5625, 0.5])
    dist = np.linalg.norm(x - contact[None, :], axis=1)
    rng = np.random.default_rng(8)
    idx = np.unique(np.concatenate([np.argsort(dist[:n])[:6], n + np.argsort(dist[n:])[:6],
                                    rng.choice(2 * n, 4, replace=False)]))
    op = oracle_operator(cell, close_targets=idx, close_rule="barycentric")
    sigma = rng.standard_normal(2 * ctx.N)
    ref = op.apply(sigma.reshape(-1, 2), targets=idx)
    for prec, tol in ((bie.BIE_FP64, 1e-10), (bie.BIE_DF64, 1e-10), (bie.BIE_MIXED, 5e-5)):
        y = ctx.apply(sigma, precision=prec).reshape(-1, 2)[idx]
        assert _rel(y, ref) < tol, (prec, _rel(y, ref))
    ctx.close()


def test_barycentric_blocks_in_a_batch_and_with_the_preconditioner():
    """The barycentric blocks of a batch are those of each cell's own context
    (FP64 applications to 1e-12, as for the fine rule: the near-sum splits
    change the rounding order), and the contact-block preconditioner
    assembled from them brings a near-contact solve to 1e-10."""
    cells = [workloads.two_ellipses(2e-3, 256),
             workloads.small_cell(n_bodies=4, nodes=128, seed=3, phi=0.3, gap=3e-3)]
    for c in cells:  # one set of proxy and collocation counts for the batch and the single contexts
        c["solver"] = dict(n_proxy=48, proxy_radius=1.5, n_coll=24, gmres_tol=1e-10)
    ctx = bie.Context(cells, precision=bie.BIE_FP64, close_rule=1)
    rng = np.random.default_rng(12)
    sigma = rng.standard_normal(2 * ctx.N)
    y = ctx.apply(sigma, precision=bie.BIE_FP64)
    no = ctx.node_offsets
    for k, c in enumerate(cells):
        s = bie.Context(c, precision=bie.BIE_FP64, close_rule=1)
        sl = slice(2 * no[k], 2 * no[k + 1])
        assert _rel(y[sl], s.apply(sigma[sl], precision=bie.BIE_FP64)) < 1e-12
        s.close()
    ctx.close()
    pc = bie.Context(workloads.two_ellipses(1e-5, 512), precision=bie.BIE_MIXED, close_rule=1, precond=1,
                     gmres_max=1000, max_refine=40)
    _, info = pc.solve()
    assert info["rel_residual"] <= 1e-10
    pc.close()


def test_barycentric_and_fine_rules_solve_alike():
    """The two close-evaluation rules are two spectrally accurate
    discretisations of the same integral (they differ in the high modes of
    the density: one interpolates sigma, the other sigma / tau).  On the two
    ellipses 2e-3 apart with 512 nodes each (resolved at that gap, the
    Sec. 8 Example 1 study), the body velocities, rotation rates and mu_eff
    agree to 1e-9 (measured 3e-11, 2e-10, 7e-11) and the densities to 1e-5
    (3e-6, concentrated at the contact)."""
    cell = workloads.two_ellipses(2e-3, 512)
    out = []
    for rule in (0, 1):
        ctx = bie.Context(cell, precision=bie.BIE_FP64, close_rule=rule)
        sig, info = ctx.solve()
        assert info["rel_residual"] <= 1e-10
        v, om, mu = ctx.velocities(sig)
        out.append((sig, v, om, mu))
        ctx.close()
    (s0, v0, o0, m0), (s1, v1, o1, m1) = out
    assert _rel(s1, s0) < 1e-5
    assert np.abs(v1 - v0).max() < 1e-9 and np.abs(o1 - o0).max() < 1e-9 and abs(m1 - m0) < 1e-9


def _errors(gap, ns, n_ref):
    from paper_1912_04501_gb300 import convergence
    ref, rows = convergence.study(gap, ns, n_ref)
    return ref, {r["n"]: max(r["err_v"], r["err_omega"]) for r in rows}, rows


def test_spectral_convergence_onset_scales_with_gap():
    """Sec. 8, Example 1: errors in v and omega against a finer solve fall
    spectrally in N, from an onset that grows like 1/sqrt(d): ~60 nodes per
    ellipse reach the solve's own accuracy at d = 1e-1 (the 1e-10 residual
    leaves ~1e-10 in omega), a few hundred are needed at 1e-3."""
    _, e1, _ = _errors(1e-1, [32, 64], 256)
    assert e1[32] > 1e-8 and e1[64] < 3e-10, e1
    _, e3, rows = _errors(1e-3, [256, 768], 2048)
    assert e3[256] > 1e-6 and e3[768] < 1e-9, e3
    assert all(r["rel_residual"] <= 1e-10 for r in rows)


def test_gap_1e5_converges():
    """d = 1e-5 (the paper's closest gap): the single-precision sweeps stall
    and the solve continues on the double-float operator, then with native
    FP64 residuals once the double-float residual reaches its own accuracy;
    every solve meets the 1e-10 tolerance and the errors fall spectrally
    (thousands of nodes per ellipse, against a reference of 4096 here)."""
    ref, e, rows = _errors(1e-5, [2048, 3072], 4096)
    assert ref["under_resolved"] == 0 and ref["rel_residual"] <= 1e-10
    assert all(r["rel_residual"] <= 1e-10 for r in rows)
    assert e[3072] < 1e-6 and e[3072] < 0.1 * e[2048], e


@pytest.mark.parametrize("gap,n,ratio", [(1e-3, 1024, 0.75), (1e-5, 2048, 0.4)])
def test_contact_preconditioner(gap, n, ratio):
    """opts.precond (right preconditioning by the dense operator block on the
    nodes in another curve's close zone): the same solution (both solves at
    the residual the gap allows; 1e-8 apart) in far fewer iterations."""
    from paper_1912_04501_gb300 import convergence
    a = convergence.solve_two_ellipses(gap, n, precond=0)
    b = convergence.solve_two_ellipses(gap, n, precond=1)
    tol = 1e-10 if gap >= 1e-3 else 3e-8
    assert a["rel_residual"] <= tol and b["rel_residual"] <= tol, (a["rel_residual"], b["rel_residual"])
    assert b["iterations"] < ratio * a["iterations"], (a["iterations"], b["iterations"])
    assert np.abs(a["omega"] - b["omega"]).max() < 1e-8 and np.abs(a["v"] - b["v"]).max() < 1e-8
