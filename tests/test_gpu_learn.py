"""GPU tests of the learned warm start: the network kernels against the
oracle's reference (oracle/mlp.py), the node features, the augmented first
GMRES cycle, and what a trained network gains.

The kernels run on the tensor cores (tcgen05): bfloat16 operands, float32
accumulation, with the roundings the oracle's bf16 mode defines.  The tests
give them weights that bfloat16 represents exactly, so the oracle (float64)
sees the same weights.  Tolerances: a node whose first-layer activations
all round to the same bfloat16 in float32 and in float64 arithmetic matches
the oracle to 1e-5 of the output scale (float32 sums of 64 products);
a node where one of them lies within 1e-6 (relative) of a rounding midpoint
may round the other way, which moves its output by at most one bfloat16
step of that activation through layers 2 and 3 (checked against that
bound).  Loss 1e-5 relative; gradient 1e-4 relative to its largest entry
(sums over 1000 nodes, where a rare rounding flip moves one term of a sum
by 2^-8 of itself).
"""
import numpy as np
import pytest

from oracle import mlp
from paper_1912_04501_gb300 import workloads

pytestmark = pytest.mark.gpu

bie = pytest.importorskip("paper_1912_04501_gb300.bie")
torch = pytest.importorskip("torch")
learn = pytest.importorskip("paper_1912_04501_gb300.learn")

F, HID = bie.BIE_NET_FEATURES, bie.BIE_NET_HIDDEN


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(mlp.n_params(F, HID)) * scale).astype(np.float32)
    return mlp.round_bf16(p)


def _data(N, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, F)).astype(np.float32)
    T = rng.standard_normal((N, 2)).astype(np.float32)
    W = rng.uniform(0.1, 1.0, N).astype(np.float32)
    return X, T, W


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _ambiguous_nodes(p, X):
    """Nodes with a first-layer activation within 1e-6 (relative) of a
    bfloat16 rounding midpoint: float32 and float64 may round it apart."""
    a1 = mlp.hidden1(p.astype(np.float64), X.astype(np.float64), HID, bf16=True)
    lo = mlp.round_bf16((a1 * (1 - 1e-6)).astype(np.float32))
    hi = mlp.round_bf16((a1 * (1 + 1e-6)).astype(np.float32))
    return (lo != hi).any(axis=1)


def test_forward_matches_oracle():
    p = _params(1)
    X, _, _ = _data(1000, 2)  # 7 full tiles of 128 and a ragged tail
    net = bie.Net()
    net.set_params(p)
    Y = torch.zeros((1000, 2), dtype=torch.float32, device="cuda")
    net.forward(_dev(X), Y)
    y = Y.cpu().numpy()
    ref = mlp.forward(p.astype(np.float64), X.astype(np.float64), HID, bf16=True)
    scale = max(1.0, np.abs(ref).max())
    amb = _ambiguous_nodes(p, X)
    assert amb.sum() < 60  # 33 of these seeded nodes
    err = np.abs(y - ref).max(axis=1)
    assert err[~amb].max() < 1e-5 * scale
    # an ambiguous node: at most one bfloat16 step (2^-8 relative) of each
    # activation, through |W3| |W2|
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p.astype(np.float64), F, HID)
    a1 = mlp.hidden1(p.astype(np.float64), X.astype(np.float64), HID, bf16=True)
    bound = (2.0 ** -8 * np.abs(a1)) @ np.abs(W2).T @ np.abs(W3).T
    assert (np.abs(y - ref)[amb] <= bound[amb] + 1e-5 * scale).all()
    # the exact (unrounded) network is a different function: the roundings are visible
    exact = mlp.forward(p.astype(np.float64), X.astype(np.float64), HID)
    assert np.abs(y - exact).max() > 1e-4 * scale
    net.close()


def test_loss_and_gradient_match_oracle():
    p = _params(3)
    X, T, W = _data(1000, 4)
    net = bie.Net()
    net.set_params(p)
    loss, g = net.loss_grad(_dev(X), _dev(T), _dev(W))
    L, gr = mlp.loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                          W.astype(np.float64), HID, bf16=True)
    assert loss == pytest.approx(L, rel=1e-5)
    assert np.abs(g - gr).max() < 1e-4 * np.abs(gr).max()
    # every parameter block on its own scale (a dropped or misplaced block fails)
    o = 0
    for k in (HID * F, HID, HID * HID, HID, 2 * HID, 2):
        assert np.abs(g[o:o + k] - gr[o:o + k]).max() < 1e-3 * np.abs(gr[o:o + k]).max(), o
        o += k
    net.close()


def test_gradient_over_many_tiles_and_ctas():
    """More tiles than CTAs: each CTA accumulates several tiles in tensor
    memory before the blocks are added."""
    p = _params(8)
    X, T, W = _data(300 * 128 + 77, 9)
    net = bie.Net()
    net.set_params(p)
    loss, g = net.loss_grad(_dev(X), _dev(T), _dev(W))
    L, gr = mlp.loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                          W.astype(np.float64), HID, bf16=True)
    assert loss == pytest.approx(L, rel=1e-5)
    assert np.abs(g - gr).max() < 1e-4 * np.abs(gr).max()
    net.close()


def test_adam_steps_match_oracle():
    p = _params(5)
    X, T, W = _data(700, 6)
    net = bie.Net()
    net.set_params(p)
    pr = p.astype(np.float64)
    m = np.zeros_like(pr)
    v = np.zeros_like(pr)
    for t in range(1, 4):
        # the reference steps from the GPU's own gradient (of the bfloat16
        # weights the kernels read), on the FP32 master weights
        _, g = net.loss_grad(_dev(X), _dev(T), _dev(W))
        net.adam_step(1e-3)
        pr, m, v = mlp.adam_step(pr, g.astype(np.float64), m, v, t, lr=1e-3)
    assert np.abs(net.get_params() - pr).max() < 1e-6


def test_features_columns():
    cell = workloads.two_ellipses(2e-3, 160)
    ctx = bie.Context(cell, precision=bie.BIE_MIXED, warm_start=1)
    X0 = ctx.features()
    x, n, w, k = ctx.nodes()
    assert X0.shape == (ctx.N, F)
    assert np.abs(X0[:, 0:2] - n).max() < 1e-6
    # no densities yet: their columns are zero
    assert np.all(X0[:, 5:9] == 0)
    # the two curves face each other across the 2e-3 gap: the nearest-curve
    # distance at the closest nodes is about the gap
    h = np.array([np.sum(w[:160]) / 160] * 160 + [np.sum(w[160:]) / 160] * 160)
    dmin = np.exp(X0[:, 9]) * h
    assert dmin.min() == pytest.approx(2e-3, rel=0.05)
    ctx.step(1e-3, 2)
    X2 = ctx.features()
    s = ctx.get_state()["sigma"].reshape(-1, 2)
    assert np.abs(X2[:, 5:7] - s).max() < 1e-5 * np.abs(s).max()  # mu = gamma = 1
    ctx.close()


@pytest.mark.parametrize("mode", [2, 3])
def test_augmented_start_meets_tolerance(mode):
    """Warm starts 2 and 3 solve to the same FP64-class tolerance as a zero
    start, and their trajectories agree with it."""
    cell = workloads.small_cell(n_bodies=4, nodes=128, seed=11, phi=0.25)
    net = bie.Net()
    net.set_params(_params(7, scale=0.05))
    runs = {}
    for m in (0, mode):
        ctx = bie.Context(cell, precision=bie.BIE_MIXED, warm_start=m)
        if m == 2:
            ctx.set_warm_net(net)
        its = []
        for _ in range(4):
            _, info = ctx.step(1e-3, 1)
            assert info["rel_residual"] <= 1e-10
            its.append(info["iterations"])
        runs[m] = (ctx.get_state(), its)
        ctx.set_warm_net(None)
        ctx.close()
    a, b = runs[0][0], runs[mode][0]
    assert np.abs(a["xc"] - b["xc"]).max() < 1e-9
    assert np.abs(a["theta"] - b["theta"]).max() < 1e-8
    net.close()


def test_trained_network_gain():
    """Train on a few small seeded suspensions, then step a held-out one from
    the same trajectory point with each start, all to the same 1e-10
    residual: the network predicts the density change better than predicting
    no change; the learned start (recycled directions + the network's)
    needs fewer iterations than a zero start and no more than 15% above the
    recycled directions alone (warm_start 3) -- the recycled directions
    already span most of a step's change, so the network's direction adds
    little on these cells (the 400- and 25-ellipse figures are in the
    design notes)."""
    def small(seed):
        c = workloads.small_cell(n_bodies=6, nodes=128, seed=seed, phi=0.3, gap=2e-2)
        return c
    X, T, W, solves = learn.generate([21, 22, 23], steps=8, cell_fn=small)
    net = bie.Net()
    net.set_params(learn.init_params(seed=0))
    res = learn.train(net, X, T, W, epochs=40, batch=2048, lr=3e-3, lr_end=3e-4)
    assert res["val_rel"] < 0.9, res
    ev = learn.evaluate(small(24), net.get_params(), steps=4, modes=(0, 3, 2))
    for m in (0, 3, 2):
        assert max(ev[m]["rel_residual"]) <= 1e-10
    print("iterations per step: zero %.1f, recycled %.1f, learned %.1f" % tuple(
        ev[m]["mean_iterations"] for m in (0, 3, 2)))
    assert ev[2]["mean_iterations"] < ev[0]["mean_iterations"], ev
    assert ev[2]["mean_iterations"] <= 1.15 * ev[3]["mean_iterations"], ev
    net.close()
