#!/usr/bin/env python
"""Benchmark of the periodized Stokes BIE hot path on one GB300 per rank.

Workload (the largest single-GPU configuration): 400 ellipses per unit cell,
area fraction 0.35, aspect ratios in [1, 3], minimum gap 2e-3, 256 nodes per
body (102400 nodes), lattice (1,0),(0,1), mu = gamma = 1, forward Euler with
dt = 1e-3 (synthetic seeded suspension).  One timed "step" is one forward-
Euler time step: solve the mobility BIE to a relative FP64-class residual of
1e-10 (single-precision pair sums inside iterative refinement with
double-float residuals; the first GMRES cycle augmented with the previous
density, its last change and the shipped warm-start network's predicted
change, the second refinement sweep with the previous step's second-sweep
correction), extract velocities and mu_eff, move the bodies, shear the
lattice and rebuild the discretisation, close-evaluation tables and proxy
fit.  Beside it: GMRES iterations per step of the three starts on the same
steps (zero, recycled directions, recycled + network), the plain FP64 solve
(zero start, double-precision pair sums) in seconds per shear time, and the
25-ellipse cell (6400 nodes) measured the same way.

value: near-image pair evaluations (9 N^2 per operator application, every
single-precision and FP64-class application counted) per second, whole job
(all ranks), in Gpairs/s.  Multi-GPU runs shard the one cell by target
(whole bodies per rank, an all-gather of the owned rows after every operator
application; strong scaling).

--impl reference times the FP64 CPU oracle (numpy, all host cores) on a
bounded sample of the targets of the same workload and reports the same
metric.
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "periodized matvec Gpairs/s; s per shear time @1e-10, mixed+learned vs plain FP64"
UNIT = "Gpairs/s"
WORKLOADS = {
    "config5": "400 ellipses/cell, phi 0.35, AR U[1,3], gap>=2e-3, 256 nodes/body (N=102400), dt 1e-3",
    "config2": "25 ellipses/cell, phi 0.3, AR U[1,3], gap>=1e-2, 256 nodes/body (N=6400), dt 1e-3",
}
# algorithmic flops of one near pair (the double-layer kernel of Eq. 3.1): the
# difference r (2), |r|^2 (3), r.n and r.q (3 + 3), their product over |r|^4
# (3, one reciprocal of |r|^2 not counted) and the accumulation of c r (4)
FLOPS_PER_PAIR = 18.0
# the same with the three images of a lattice row sharing r_y, r_y^2, r_y n_y
# and r_y q_y (4 flops per row of 3 pairs): the row-shared kernel k_near32r
FLOPS_PER_PAIR_ROWS = 14.0 + 4.0 / 3.0
# FP32 instructions per pair of k_near32r (an FMA counts once): the FP32
# pipe's issue limit is half the FMA flop peak in these units
OPS_PER_PAIR_ROWS = 9.0 + 4.0 / 3.0
# the doubled-cell kernel shares the r_y terms between a node's two images
# at one lattice row (dm = 0, 1): 14 per pair + 4 per two pairs
FLOPS_PER_PAIR_UROWS = 14.0 + 4.0 / 2.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="config5", choices=sorted(WORKLOADS))
    p.add_argument("--images", type=int, default=9, choices=[9, 4],
                   help="periodizer of the timed context: 9 = 3x3 images of every body (the headline), 4 = the "
                        "paper's doubled cell (four images per node)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batch", action="store_true", help="skip the 64-cell ensemble's extra key")
    p.add_argument("--mixed-only", action="store_true",
                   help="time the mixed-precision steps only (no comparisons, no end-to-end loop); "
                        "used for kernel launch lists")
    return p.parse_args()


def make_cell(name):
    from paper_1912_04501_gb300 import workloads
    return getattr(workloads, name)()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and self.uuid not in parts[1]:
                continue
            rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        hi = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(hi) if hi else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _function_text(text, name, qualifier):
    """The definition of function `name` whose declaration carries
    `qualifier` (with a template line just above it), or ""."""
    import re
    for m in re.finditer(r"\b%s\s*\(" % re.escape(name), text):
        q = text.rfind(qualifier, 0, m.start())
        if q < 0 or any(ch in text[q:m.start()] for ch in ";{}"):
            continue
        i, depth = m.end() - 1, 0
        while i < len(text):
            depth += {"(": 1, ")": -1}.get(text[i], 0)
            if depth == 0:
                break
            i += 1
        j = i + 1
        while j < len(text) and text[j] in " \t\n":
            j += 1
        if j >= len(text) or text[j] != "{":
            continue  # a declaration or a call, not the definition
        k, depth = j, 0
        while k < len(text):
            depth += {"{": 1, "}": -1}.get(text[k], 0)
            if depth == 0:
                break
            k += 1
        start = text.rfind("\n", 0, q) + 1
        prev = text.rfind("\n", 0, max(0, start - 1)) + 1
        if text[prev:start].lstrip().startswith("template"):
            start = prev
        return text[start:k + 1]
    return ""


def kernel_source(kernel):
    """Source text of a kernel in the library and of the library's device
    functions it calls (directly or through others), the unit the committed
    ncu summaries are keyed on."""
    import glob
    import re
    texts = [open(p).read() for p in sorted(glob.glob(os.path.join(ROOT, "paper_1912_04501_gb300", "csrc", "*.c*")))]
    for text in texts:
        body = _function_text(text, kernel, "__global__")
        if body:
            seen, todo, helpers = {kernel}, [body], []
            while todo:  # device functions it calls, and theirs
                for name in sorted(set(re.findall(r"\b([a-z][a-z0-9_]*)\s*(?:<[^<>;]*>)?\s*\(", todo.pop()))):
                    if name in seen:
                        continue
                    seen.add(name)
                    for t in texts:
                        h = _function_text(t, name, "__device__")
                        if h:
                            helpers.append(h)
                            todo.append(h)
                            break
            return body + "".join(sorted(helpers))
    return ""


def source_hash(kernel):
    return hashlib.sha256(kernel_source(kernel).encode()).hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of
    this workload, if it was taken on the kernel's current source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ": " in line and line.startswith("- "):
            k, v = line[2:].split(": ", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel source sha256[:16]") != source_hash(kernel):
        return None
    try:
        return float(vals["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
_OP = None


def _oracle_init(cell, close_targets):
    global _OP
    from oracle import bie as obie
    from oracle import geometry
    s = geometry.Suspension(cell["e1"], cell["e2"], cell["centre"], cell["mu"], cell["gamma"], cell["bodies"])
    sv = cell["solver"]
    _OP = obie.Operator(s, n_proxy=sv["n_proxy"], proxy_radius=sv["proxy_radius"], n_coll=sv["n_coll"],
                        close_targets=close_targets)


def _oracle_apply(args):
    sigma, idx = args
    t0 = time.perf_counter()
    _OP.apply(sigma, targets=idx)
    return time.perf_counter() - t0


class OracleSample:
    """The FP64 oracle's operator application at a bounded sample of the
    targets of a workload, on one core (in process) or on `procs` cores
    (spawned workers, each with its own share of the sample; the wall time of
    the whole application is what counts)."""

    def __init__(self, cell, procs, per_proc, seed=0):
        import numpy as np
        self.N = sum(b["n"] for b in cell["bodies"])
        rng = np.random.default_rng(seed)
        self.idx = np.sort(rng.choice(self.N, min(self.N, procs * per_proc), replace=False))
        self.sigma = rng.standard_normal((self.N, 2))
        self.procs = procs
        self.chunks = np.array_split(self.idx, procs)
        if procs == 1:
            _oracle_init(cell, self.idx)
            self.pool = None
        else:
            self.pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_init, initargs=(cell, self.idx))
            self.pool.map(_oracle_apply, [(self.sigma, c[:1]) for c in self.chunks])  # workers ready

    def run(self):
        t0 = time.perf_counter()
        if self.pool is None:
            _oracle_apply((self.sigma, self.idx))
        else:
            self.pool.map(_oracle_apply, [(self.sigma, c) for c in self.chunks])
        dt = time.perf_counter() - t0
        pairs = 9.0 * len(self.idx) * self.N
        return pairs / dt / 1e9, dt

    def describe(self, dt):
        return (f"FP64 numpy oracle, {self.procs} process(es): one operator application evaluated at "
                f"{len(self.idx)} of {self.N} sampled targets ({9.0 * len(self.idx) * self.N:.3g} near pairs, plus "
                f"each process's full wall discrepancy, proxy fit and close pairs of its targets), {dt:.1f} s")

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()


def cpu_baselines(cell, per_proc_single=96, per_proc_all=48):
    """Single-core and all-core oracle rates (Gpairs/s) on bounded samples."""
    out = {}
    one = OracleSample(cell, 1, per_proc_single)
    v, dt = one.run()
    out["single"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": one.describe(dt)}
    one.close()
    n = os.cpu_count() or 1
    if n > 1:
        allc = OracleSample(cell, n, per_proc_all, seed=1)
        v, dt = allc.run()
        out["all"] = {"value": v, "unit": UNIT, "cores": n, "kind": "oracle", "sample": allc.describe(dt)}
        allc.close()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    cell = make_cell(args.workload)
    procs = os.cpu_count() or 1
    smp = OracleSample(cell, procs, 16)
    vals, secs = [], []
    for k in range(args.warmup + args.steps):
        v, dt = smp.run()
        if k >= args.warmup:
            vals.append(v)
            secs.append(dt)
    smp.close()
    v = statistics.mean(vals)
    desc = smp.describe(statistics.mean(secs))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "step": "one oracle application at a bounded sample of the targets", "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
def whole_job(units, ms, dist, device, shared=False):
    """Whole-job figures over the ranks: the slowest rank's time (max) and
    the units -- summed over independent replicas, or (shared) those of the
    one problem all ranks solve together (every rank counts the same units,
    taken from rank 0).  dist None: one process."""
    if dist is None:
        return float(units), float(ms)
    import torch
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if shared:
        dist.broadcast(u, 0)
    else:
        dist.all_reduce(u)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u[0]), float(t[0])


def timed_steps(ctx, stream, dt, steps, flush=None):
    """Per-step device times (CUDA events on the context's stream, L2
    flushed before each step) and solve statistics of `steps` time steps."""
    import numpy as np
    import torch
    out = dict(ms=[], applies32=0, applies64=0, iters=[], mu=[])
    for _ in range(steps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m, info = ctx.step(dt, 1)
        e1.record(stream)
        e1.synchronize()
        out["ms"].append(e0.elapsed_time(e1))
        out["applies32"] += info["applies32"]
        out["applies64"] += info["applies64"]
        out["iters"].append(info["iterations"])
        out["mu"].append(float(np.ravel(m)[0]))  # a batch returns one value per cell
    return out


def restore(bie, cell, st, stream, **kw):
    c = bie.Context(cell, precision=bie.BIE_MIXED, **kw)
    c.set_stream(stream.cuda_stream)
    c.set_state(st["t"], st["e2"], st["xc"], st["theta"], st["sigma"], st["sigma_prev2"], st["dt_prev"], st["d2"])
    return c


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    from paper_1912_04501_gb300 import bie, learn, workloads

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    name = args.workload
    cell = make_cell(name)
    dt = cell["dt"]
    N = sum(b["n"] for b in cell["bodies"])
    nb = len(cell["bodies"])
    pairs_per_apply = float(args.images) * N * N
    img_opts = dict(n_images=4, n_proxy=128, n_coll=32) if args.images == 4 else {}
    stream = torch.cuda.Stream()
    net = learn.default_net(device=local)
    mode = 2 if net is not None else 3
    # the default near-sum tile shape: fixed, so that a profiler run of this
    # command launches the same kernels as the timed one (the autotuner's
    # choice depends on timings, which a profiler distorts); direct launches
    # (replaying captured graphs measured no faster)
    ctx = bie.Context(cell, precision=bie.BIE_MIXED, device=local, warm_start=mode, autotune=0, graph=0, **img_opts)
    shape, _ = ctx.near_shape()
    # the packed shapes share each lattice row's r_y when e1 = (L1, 0), as in
    # every sheared cell here
    rows = bool(bie.NEAR32_SHAPES[shape][0]) and cell["e1"][1] == 0.0 and args.images == 9
    near32 = "k_near32r" if rows else ("k_near32x2" if bie.NEAR32_SHAPES[shape][0] else "k_near32")
    if args.images == 4:
        near32 = "k_near32u"
    fpp32 = FLOPS_PER_PAIR_ROWS if rows else FLOPS_PER_PAIR
    ctx.set_stream(stream.cuda_stream)
    if net is not None:
        net.set_stream(stream.cuda_stream)
        ctx.set_warm_net(net)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    sharded = None
    if world > 1:
        # one cell solved by all ranks: each owns the targets of whole bodies
        # and all-gathers its rows after every operator application
        from paper_1912_04501_gb300 import shard
        sharded = shard.ShardedSolve(ctx, [b["n"] for b in cell["bodies"]], rank, world)

    for _ in range(args.warmup):
        ctx.step(dt, 1)
    torch.cuda.synchronize()
    st0 = ctx.get_state()  # the trajectory point the start comparison restarts from
    props = torch.cuda.get_device_properties(local)
    uuid = str(getattr(props, "uuid", "") or "")
    ctx.profile_read()
    ctx.profile(True)
    barrier()
    clocks = Clocks(uuid)
    t_wall = time.perf_counter()
    run = timed_steps(ctx, stream, dt, args.steps, flush)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    prof = ctx.profile_read()
    ctx.profile(False)
    total_ms = sum(run["ms"])
    applies32, applies64 = run["applies32"], run["applies64"]
    pairs = pairs_per_apply * (applies32 + applies64)  # applies64: FP64-class (double-float) residuals
    # whole job: the cell's pairs / slowest rank's time
    pairs_all, t_ms = whole_job(pairs, total_ms, dist, "cuda", shared=True)
    value = pairs_all / (t_ms / 1e3) / 1e9
    ms_per_step = t_ms / args.steps

    if world > 1:
        # sharded runs report the timed steps only (the comparisons below are
        # single-GPU measurements)
        if rank == 0:
            print(json.dumps({
                "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOADS[name], "N": N, "bodies": nb,
                           "parallelism": f"target-sharded over {world} GPUs: whole bodies per rank, one all-gather "
                                          f"of the owned rows per operator application",
                           "l2": "flushed between timed steps (256 MB write)"},
                "s_per_shear_time": ms_per_step / 1e3 / dt, "gpu_launches": prof["launches"], "clocks": clk,
                "e2e": None}), flush=True)
        sharded.close()
        ctx.set_warm_net(None)
        ctx.close()
        dist.destroy_process_group()
        return

    if args.mixed_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": ms_per_step, "mixed_only": True,
                              "config": {"workload": WORKLOADS[name]},
                              "gpu_launches": prof["launches"], "profile": prof}), flush=True)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return

    # GMRES iterations and wall time per step of the three starts, on the same
    # three steps from the same trajectory point (state and history restored)
    starts = {}
    for m, label in ((0, "zero"), (3, "recycled"), (mode, "learned" if mode == 2 else "recycled (no network)")):
        if label in starts:
            continue
        cm = restore(bie, cell, st0, stream, device=local, warm_start=m)
        if m == 2:
            cm.set_warm_net(net)
        r = timed_steps(cm, stream, dt, 3)
        starts[label] = {"iterations": r["iters"], "ms": r["ms"]}
        if m == 2:
            cm.set_warm_net(None)
        cm.close()

    # the paper's own periodizer (four images per node inside the doubled
    # cell, proxies on its walls): the same steps with 4 N^2 near pairs per
    # application instead of 9 N^2
    cu = bie.Context(cell, precision=bie.BIE_MIXED, device=local, warm_start=mode, n_images=4, n_proxy=128,
                     n_coll=32)
    cu.set_stream(stream.cuda_stream)
    if net is not None:
        cu.set_warm_net(net)
    for _ in range(max(3, args.warmup)):
        cu.step(dt, 1)
    cu.profile_read()
    cu.profile(True)
    ru = timed_steps(cu, stream, dt, max(3, args.steps // 4), flush)
    pu = cu.profile_read()
    cu.profile(False)
    if net is not None:
        cu.set_warm_net(None)
    cu.close()
    pairs_u = 4.0 * N * N
    msu = statistics.mean(ru["ms"])
    utilde = {"workload": WORKLOADS[name] + "; doubled-cell periodizer: 4 images per node, 128 proxies on the "
                                            "doubled cell's walls, 32 collocation points per wall",
              "steps": len(ru["ms"]), "ms_per_step": msu, "s_per_shear_time": msu / 1e3 / dt,
              "pairs_per_apply": pairs_u,
              "value": pairs_u * (ru["applies32"] + ru["applies64"]) / (sum(ru["ms"]) / 1e3) / 1e9,
              "iterations_mean": statistics.mean(ru["iters"]), "mu_eff_last": ru["mu"][-1],
              "near32_ms_per_launch": pu["near32_ms"] / max(1, pu["near32_launches"]),
              "neardf_ms_per_launch": pu["neardf_ms"] / max(1, pu["neardf_launches"]),
              "near32_tflops": (FLOPS_PER_PAIR_UROWS if cell["e1"][1] == 0.0 else FLOPS_PER_PAIR) * pairs_u
              / (pu["near32_ms"] / max(1, pu["near32_launches"]) / 1e3) / 1e12 if pu["near32_launches"] else None}

    # plain FP64 solve (zero start, double-precision pair sums): one operator
    # application timed on the device, times the plain GMRES iterations plus
    # one residual application.  The iterations are counted on the
    # double-float operator (plain GMRES, zero start, same tolerance), which
    # agrees with the FP64 one to ~1e-13 and takes the same iterations at a
    # seventh of the time; small cells run the FP64 steps themselves.
    ctx64 = bie.Context(cell, precision=bie.BIE_FP64, device=local, warm_start=0)
    ctx64.set_stream(stream.cuda_stream)
    sig = torch.randn(2 * N, dtype=torch.float64, device="cuda")
    y64 = torch.empty_like(sig)
    torch.cuda.synchronize()
    ctx64.apply(sig, y64, precision=bie.BIE_FP64)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ctx64.apply(sig, y64, precision=bie.BIE_FP64)
    ev1.record(stream)
    ev1.synchronize()
    ms64_apply = ev0.elapsed_time(ev1)
    fp64 = None
    if N > 20000:
        cdf = bie.Context(cell, precision=bie.BIE_DF64, device=local, warm_start=0)
        cdf.set_stream(stream.cuda_stream)
        cdf.set_state(st0["t"], st0["e2"], st0["xc"], st0["theta"])
        _, idf = cdf.solve()
        cdf.close()
        fp64 = {"ms_per_apply": ms64_apply, "iterations_per_step": idf["iterations"],
                "s_per_shear_time": (idf["iterations"] + 1) * ms64_apply / 1e3 / dt,
                "how": "extrapolated: one FP64 operator application (CUDA events) x (iterations of a plain zero-start "
                       "GMRES solve at the same geometry and tolerance, counted on the double-float operator, + 1 "
                       "residual application)"}
    else:  # small cells: a full plain FP64 step is measured
        ctx64.step(dt, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info64 = ctx64.step(dt, 2)
        torch.cuda.synchronize()
        fp64 = {"ms_per_apply": ms64_apply, "iterations_per_step": info64["iterations"],
                "s_per_shear_time": (time.perf_counter() - t0) / 2 / dt, "how": "measured: two plain FP64 steps"}
    ctx64.close()

    # end to end through the public API with host buffers: the state (and the
    # warm-start history) in from pinned host memory, one step, the state out
    st = ctx.get_state()
    host_in = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
               (("e2", st["e2"]), ("xc", st["xc"].ravel()), ("theta", st["theta"]), ("sigma", st["sigma"]),
                ("sigma_prev2", st["sigma_prev2"]), ("d2", st["d2"]))}
    e2e_steps = max(3, args.steps // 4)
    e2e_pairs = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.set_state(st["t"], host_in["e2"].numpy(), host_in["xc"].numpy(), host_in["theta"].numpy(),
                      host_in["sigma"].numpy(), host_in["sigma_prev2"].numpy(), st["dt_prev"],
                      host_in["d2"].numpy())
        m, info = ctx.step(dt, 1)
        out = ctx.get_state()
        e2e_pairs += pairs_per_apply * (info["applies32"] + info["applies64"])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = (3 * nb + 2 + 3 * 2 * N) * 8   # centroids, angles, e2, density, previous density, sweep correction
    d2h = (8 * nb + 3 * 2 * N + 1) * 8  # body table, density, previous density, sweep correction, mu_eff
    sms = ctx.device_sms()
    ctx.set_warm_net(None)
    ctx.close()

    # the 25-ellipse cell, measured the same way (an extra key)
    small = None
    if name != "config2":
        c2 = make_cell("config2")
        N2 = sum(b["n"] for b in c2["bodies"])
        cx = bie.Context(c2, precision=bie.BIE_MIXED, device=local, warm_start=mode)
        cx.set_stream(stream.cuda_stream)
        if net is not None:
            cx.set_warm_net(net)
        for _ in range(5):
            cx.step(c2["dt"], 1)
        r2 = timed_steps(cx, stream, c2["dt"], 10, flush)
        cx.set_warm_net(None)
        cx.close()
        c64 = bie.Context(c2, precision=bie.BIE_FP64, device=local, warm_start=0)
        c64.set_stream(stream.cuda_stream)
        c64.step(c2["dt"], 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c64.step(c2["dt"], 2)
        torch.cuda.synchronize()
        s64 = (time.perf_counter() - t0) / 2 / c2["dt"]
        c64.close()
        ms2 = statistics.mean(r2["ms"])
        small = {"workload": WORKLOADS["config2"], "ms_per_step": ms2, "s_per_shear_time": ms2 / 1e3 / c2["dt"],
                 "s_per_shear_time_fp64": s64,
                 "value": 9.0 * N2 * N2 * (r2["applies32"] + r2["applies64"]) / (sum(r2["ms"]) / 1e3) / 1e9,
                 "iterations_mean": statistics.mean(r2["iters"])}

    # the 64-cell ensemble (uneven cells in one context; its near sums from the
    # persistent work queue), measured the same way: an extra key
    batch = None
    if world == 1 and not args.no_batch:
        cells4 = workloads.config4()
        N4 = sum(sum(b["n"] for b in c["bodies"]) for c in cells4)
        pairs4 = sum(9.0 * sum(b["n"] for b in c["bodies"]) ** 2 for c in cells4)
        # the ensemble as specified: the single-precision applications replayed
        # from captured CUDA graphs, the near-sum tile shape picked by the
        # autotuner
        cb = bie.Context(cells4, precision=bie.BIE_MIXED, device=local, warm_start=mode, graph=1, autotune=1)
        cb.set_stream(stream.cuda_stream)
        if net is not None:
            cb.set_warm_net(net)
        for _ in range(3):
            cb.step(cells4[0]["dt"], 1)
        r4 = timed_steps(cb, stream, cells4[0]["dt"], 5, flush)
        # full applications (every cell active; in a lockstep solve the
        # converged cells drop out of the later launches)
        sig4 = torch.zeros(2 * N4, dtype=torch.float64, device="cuda")
        sig4.copy_(torch.from_numpy(cb.rhs()))
        out4 = torch.empty_like(sig4)
        with torch.cuda.stream(stream):
            for _ in range(3):
                cb.apply(sig4, out4, precision=bie.BIE_MIXED)
        shape4, ms_shapes4 = cb.near_shape()
        cb.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(10):
                cb.apply(sig4, out4, precision=bie.BIE_MIXED)
            e1.record(stream)
        e1.synchronize()
        p4 = cb.profile_read()
        cb.profile(False)
        cb.set_warm_net(None)
        cb.close()
        ms4 = statistics.mean(r4["ms"])
        ms4_near = p4["near32_ms"] / max(1, p4["near32_launches"])
        batch = {"workload": "64 cells, 5-50 ellipses each, phi U[0.1, 0.4], AR U[1,3], gap>=1e-2, 128-256 "
                             "nodes/body (N=%d), dt 1e-3, mixed+learned, lockstep solves" % N4,
                 "ms_per_step": ms4, "iterations_mean": statistics.mean(r4["iters"]),
                 "pairs_per_apply": pairs4,
                 "apply_ms": e0.elapsed_time(e1) / 10, "near32_ms_per_launch": ms4_near,
                 "value": pairs4 / (ms4_near / 1e3) / 1e9 if p4["near32_launches"] else None,
                 "unit": "Gpairs/s (near sum of a full application, every cell active)",
                 "near_sum": "persistent work queue (k_near32r_queue), items sorted longest first",
                 "graph": True, "tile_shape": {"chosen": shape4, "ms_per_shape": ms_shapes4}}

    # rooflines: measured CUDA-core FMA throughput of this device
    peak = bie.alu_peak(local, stream.cuda_stream)
    fp32_peak = max(peak["ffma"], peak["ffma2"])
    fp32_src = (f"measured FP32 FMA throughput of this GPU (bie_alu_peak: scalar FFMA {peak['ffma']:.1f}, packed "
                f"FFMA2 {peak['ffma2']:.1f} TFLOP/s; the larger is the peak), {sms} SMs queried")
    n32, n64, ndf = prof["near32_launches"], prof["near64_launches"], prof["neardf_launches"]
    ms32 = prof["near32_ms"] / max(1, n32)
    msdf = prof["neardf_ms"] / max(1, ndf)
    roof32 = {"kernel": near32, "bound": "alu", "unit": "TFLOP/s", "peak": fp32_peak,
              "achieved": fpp32 * pairs_per_apply / (ms32 / 1e3) / 1e12 if n32 else None,
              "flops_per_pair": fpp32, "launch_ms": ms32, "launches": n32, "device_ms_total": prof["near32_ms"],
              "peak_source": fp32_src, "traffic": profiled_traffic(near32, name)}
    if rows and n32:
        # the same launches as a fraction of the FP32 pipe's instruction rate
        roof32["fp32_issue_frac"] = OPS_PER_PAIR_ROWS * pairs_per_apply / (ms32 / 1e3) / 1e12 / (fp32_peak / 2)
    # double-float pairs run on the FP32 pipe: measured against the FP32 peak,
    # counting the same algorithmic flops per pair as the single-precision
    # kernel (the extra ~100 FP32 instructions per pair are the price of the
    # 48-bit arithmetic)
    roofdf = {"kernel": "k_near_df", "bound": "alu", "unit": "TFLOP/s", "peak": fp32_peak,
              "achieved": fpp32 * pairs_per_apply / (msdf / 1e3) / 1e12 if ndf else None,
              "launch_ms": msdf, "launches": ndf, "device_ms_total": prof["neardf_ms"],
              "peak_source": fp32_src, "traffic": profiled_traffic("k_near_df", name)}
    roof64 = {"kernel": "k_near64 (plain FP64 operator, whole application)", "bound": "alu", "unit": "TFLOP/s",
              "peak": peak["dfma"], "achieved": FLOPS_PER_PAIR * pairs_per_apply / (ms64_apply / 1e3) / 1e12,
              "launch_ms": ms64_apply, "launches": 1, "device_ms_total": ms64_apply,
              "peak_source": f"measured FP64 FMA throughput of this GPU (bie_alu_peak: {peak['dfma']:.2f} TFLOP/s)",
              "traffic": None}
    for r in (roof32, roofdf, roof64):
        r["frac"] = r["achieved"] / r["peak"] if r["achieved"] and r["peak"] else None
    ranked = sorted([roof32, roofdf], key=lambda r: -r["device_ms_total"])
    dom, other = ranked[0], [r for r in ranked[1:] if r["launches"]] + [roof64]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(cell)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[name], "N": N, "bodies": nb,
                       "precision": "FP32 pair sums; refinement residual with double-float pair sums",
                       "gmres_tol": 1e-10,
                       "warm_start": ("learned: first GMRES cycle augmented with the previous density, its last "
                                      "change and the shipped network's predicted change; second refinement sweep "
                                      "augmented with the previous step's second-sweep correction" if mode == 2 else
                                      "first GMRES cycle augmented with the previous density and its last change; "
                                      "second sweep with the previous second-sweep correction"),
                       "l2": "flushed between timed steps (256 MB write)",
                       "near_tile": {"shape": shape, "packed": bool(bie.NEAR32_SHAPES[shape][0]),
                                     "targets_per_thread": bie.NEAR32_SHAPES[shape][1],
                                     "ctas_per_sm": bie.NEAR32_SHAPES[shape][2]},
                       "sms": sms, "parallelism": "one GPU"},
            "s_per_shear_time": ms_per_step / 1e3 / dt,
            "s_per_shear_time_fp64": fp64["s_per_shear_time"],
            "fp64_plain": fp64,
            # operator applications per second (all ranks), and the pairs of an
            # application outside the near sum: wall discrepancy (2m wall
            # points x the 6 far image rows/columns of every node, velocity
            # and traction) and proxy correction (every node x M proxies)
            "matvecs_per_s": (applies32 + applies64) / (t_ms / 1e3),
            "pairs_per_apply": {"near": pairs_per_apply,
                                "wall": 2.0 * cell["solver"]["n_coll"] * 6 * N,
                                "proxy": float(N * cell["solver"]["n_proxy"])},
            "solve": {"applies32": applies32, "applies64": applies64,
                      "iterations_mean": statistics.mean(run["iters"]), "mu_eff_last": run["mu"][-1],
                      "starts_same_steps": starts},
            "roofline": {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")},
            "roofline_detail": [dom] + other,
            "alu_peaks_tflops": peak,
            "cpu_baseline": cpu["all"] if cpu and "all" in cpu else (cpu or {}).get("single"),
            "cpu_baseline_single_core": (cpu or {}).get("single"),
            "e2e": {"value": e2e_pairs / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps},
            "config2": small,
            "config4": batch,
            "utilde": utilde,
            "gpu_launches": prof["launches"],
            "clocks": clk,
            "wall_s_timed": t_wall,
        }
        print(json.dumps(line), flush=True)
    if net is not None:
        net.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
