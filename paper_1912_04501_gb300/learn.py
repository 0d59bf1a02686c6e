"""Training and evaluation of the warm-start network (include/bie.h, "Learned
warm start").

The network is trained on densities the solver itself produces: suspensions
shaped like the 25-ellipse cell (seeded placements distinct from the
evaluation seeds) are stepped forward in time; before every step the node
features of the context are recorded (bie_features), after it the converged
density, and the training target is the density change over the step in
units of mu |gamma| dt (or, with --target second, the part of it beyond the
linear extrapolation of the last two densities).  The loss weights each node by its quadrature weight,
so that it measures the change in the L2 norm on the curves.

All arithmetic runs in the library's kernels (features, forward, gradient,
Adam); this module only moves data.  Dataset tensors live on the GPU; each
minibatch is a slice of a per-epoch permutation.
"""
import argparse
import math
import os
import time

import numpy as np

from . import bie, workloads

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_PARAMS = os.path.join(HERE, "warm_net_params.npy")

# The shipped network: trained by `python -m paper_1912_04501_gb300.learn`
# with these settings (seeds distinct from the evaluation cells' seeds).
TRAIN_SEEDS = list(range(100, 112))
TRAIN_STEPS = 20
TRAIN = dict(epochs=30, batch=8192, lr=2e-3, lr_end=1e-4, seed=0)
TARGET = "change"


def init_params(n_in=bie.BIE_NET_FEATURES, hidden=bie.BIE_NET_HIDDEN, seed=0, out_scale=1e-2):
    """Glorot-uniform hidden layers, a small output layer (the initial
    prediction is near zero), zero biases; one flat float32 vector."""
    rng = np.random.default_rng(seed)

    def glorot(o, i, s=1.0):
        a = s * math.sqrt(6.0 / (i + o))
        return rng.uniform(-a, a, (o, i))

    parts = [glorot(hidden, n_in), np.zeros(hidden), glorot(hidden, hidden), np.zeros(hidden),
             glorot(2, hidden, out_scale), np.zeros(2)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def training_cell(seed, n_bodies=25, phi=0.3, nodes=256, gap=1e-2):
    """A suspension shaped like the 25-ellipse cell (area fraction 0.3, aspect
    ratios in [1, 3], minimum gap 1e-2, 256 nodes per body), seeded."""
    cell = workloads.random_cell(n_bodies, phi, (1.0, 3.0), gap, nodes, seed)
    cell.update(solver=dict(n_proxy=48, proxy_radius=1.5, n_coll=24, gmres_tol=1e-10), dt=1e-3)
    return cell


def generate(seeds, steps, dt=1e-3, lead=2, cell_fn=training_cell, log=None, target=None):
    """Run each seeded cell `lead` steps (so two earlier densities exist),
    then record `steps` (features, target, weight) triples.  Returns host
    arrays X (M x F float32), T (M x 2 float32), W (M float32) and the number
    of solves.  target "change" (default TARGET): the density change over the
    step; "second": the change beyond the linear extrapolation of the last
    two densities, sigma_{n+1} - sigma_n - (sigma_n - sigma_{n-1}) dt / dt_prev,
    the part of the new density the recycled directions (sigma_n and its last
    change) do not span; both in units of mu |gamma| dt."""
    target = target or TARGET
    Xs, Ts, Ws = [], [], []
    solves = 0
    for seed in seeds:
        cell = cell_fn(seed)
        ctx = bie.Context(cell, precision=bie.BIE_MIXED, warm_start=1)
        scale = cell["mu"] * abs(cell["gamma"]) * dt
        ctx.step(dt, lead)
        for _ in range(steps):
            X = ctx.features()
            w = ctx.nodes()[2]
            st = ctx.get_state()
            s0 = st["sigma"]
            ctx.step(dt, 1)
            s1 = ctx.get_state()["sigma"]
            d = s1 - s0
            if target == "second":
                d = d - (s0 - st["sigma_prev2"]) * (dt / st["dt_prev"])
            Xs.append(X)
            Ts.append((d / scale).reshape(-1, 2).astype(np.float32))
            Ws.append(w.astype(np.float32))
            solves += 1
        ctx.close()
        if log:
            log(f"seed {seed}: {solves} solves recorded")
    return np.concatenate(Xs), np.concatenate(Ts), np.concatenate(Ws), solves


def train(net, X, T, W, epochs=20, batch=8192, lr=2e-3, lr_end=2e-4, seed=0, val_frac=0.1, log=None):
    """Adam on minibatches; the last val_frac of the rows (whole solves, as
    generated) is held out.  Returns a dict with the loss history and the
    held-out loss relative to predicting zero change."""
    import torch
    dev = torch.device("cuda")
    M = X.shape[0]
    mv = int(M * (1.0 - val_frac))
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    Td = torch.from_numpy(np.ascontiguousarray(T)).to(dev)
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(dev)
    Xv, Tv, Wv = Xd[mv:].contiguous(), Td[mv:].contiguous(), Wd[mv:].contiguous()
    zero_v = float((Wv * (Tv * Tv).sum(1)).sum() / Wv.sum())
    gen = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    steps_per_epoch = max(1, mv // batch)
    total = epochs * steps_per_epoch
    k = 0
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(mv, generator=gen).to(dev)
        for b in range(steps_per_epoch):
            idx = perm[b * batch:(b + 1) * batch]
            xb, tb, wb = Xd[idx].contiguous(), Td[idx].contiguous(), Wd[idx].contiguous()
            loss, _ = net.loss_grad(xb, tb, wb, with_grad=False)
            frac = k / max(1, total - 1)
            net.adam_step(lr * (lr_end / lr) ** frac)
            k += 1
        vloss, _ = net.loss_grad(Xv, Tv, Wv, with_grad=False)
        hist.append((ep, loss, vloss))
        if log:
            log(f"epoch {ep}: train {loss:.4g} held-out {vloss:.4g} (zero predictor {zero_v:.4g}) "
                f"{time.time() - t0:.1f}s")
    return dict(history=hist, val_loss=hist[-1][2], zero_loss=zero_v, val_rel=hist[-1][2] / zero_v,
                train_rows=mv, val_rows=M - mv, seconds=time.time() - t0)


def evaluate(cell, params, steps, dt=1e-3, lead=2, modes=(0, 1, 3, 2), precision=bie.BIE_MIXED):
    """Iterations and wall time per step for each warm-start mode on the same
    trajectory start: 0 zero start, 1 previous density as the guess, 3
    augmentation by the previous density and its change, 2 the same plus the
    network's prediction.  Every run solves to the same FP64-class residual
    tolerance (gmres_tol), so the counts compare at equal final residual."""
    import torch
    net = bie.Net()
    net.set_params(params)
    out = {}
    for mode in modes:
        ctx = bie.Context(cell, precision=precision, warm_start=mode)
        if mode == 2:
            ctx.set_warm_net(net)
        ctx.step(dt, lead)
        its, a32, a64, res, secs = [], [], [], [], []
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = ctx.step(dt, 1)
            torch.cuda.synchronize()
            secs.append(time.perf_counter() - t0)
            its.append(info["iterations"])
            a32.append(info["applies32"])
            a64.append(info["applies64"])
            res.append(info["rel_residual"])
        out[mode] = dict(iterations=its, applies32=a32, applies64=a64, rel_residual=res, seconds=secs,
                         mean_iterations=float(np.mean(its)), mean_seconds=float(np.mean(secs)))
        ctx.set_warm_net(None)
        ctx.close()
    net.close()
    return out


def load_params(path=DEFAULT_PARAMS):
    """The shipped (or a saved) parameter vector, float32."""
    return np.load(path).astype(np.float32)


def default_net(device=0):
    """A Net holding the shipped parameters, or None if there are none."""
    if not os.path.exists(DEFAULT_PARAMS):
        return None
    net = bie.Net(device=device)
    net.set_params(load_params())
    return net


def main():
    ap = argparse.ArgumentParser(description="train the warm-start network on solver-generated densities, or "
                                             "compare the warm starts on a workload (--evaluate)")
    ap.add_argument("--out", default=DEFAULT_PARAMS)
    ap.add_argument("--seeds", type=int, nargs="*", default=TRAIN_SEEDS)
    ap.add_argument("--steps", type=int, default=TRAIN_STEPS)
    ap.add_argument("--epochs", type=int, default=TRAIN["epochs"])
    ap.add_argument("--evaluate", nargs="*", default=None,
                    help="workloads (e.g. config2 config5) on which to compare the starts with --params")
    ap.add_argument("--params", default=DEFAULT_PARAMS)
    ap.add_argument("--eval-steps", type=int, default=10)
    ap.add_argument("--target", choices=("change", "second"), default=TARGET)
    a = ap.parse_args()
    if a.evaluate is not None:
        import json
        for name in a.evaluate:
            ev = evaluate(getattr(workloads, name)(), load_params(a.params), a.eval_steps, modes=(3, 2))
            print(json.dumps({"workload": name, "params": os.path.basename(a.params), "steps": a.eval_steps,
                              "recycled": ev[3], "learned": ev[2]}), flush=True)
        return
    X, T, W, solves = generate(a.seeds, a.steps, log=print, target=a.target)
    net = bie.Net()
    net.set_params(init_params(seed=0))
    res = train(net, X, T, W, log=print, **dict(TRAIN, epochs=a.epochs))
    np.save(a.out, net.get_params())
    print(f"{solves} solves, {X.shape[0]} nodes; held-out loss / zero predictor = {res['val_rel']:.3g}; "
          f"wrote {a.out}")
    net.close()


if __name__ == "__main__":
    main()
