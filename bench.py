#!/usr/bin/env python
"""Benchmark of the periodized Stokes BIE hot path on one GB300 per rank.

Workload: 25 equal-area ellipses per unit cell, area fraction 0.3, aspect
ratios in [1, 3], minimum gap 1e-2, 256 nodes per body (6400 nodes), lattice
(1,0),(0,1), mu = gamma = 1, forward Euler with dt = 1e-3 (synthetic seeded
suspension).  One timed "step" is one forward-Euler time step: solve the
mobility BIE to a relative FP64-class residual of 1e-10 (single-precision
pair sums inside iterative refinement with double-float residuals; the first
GMRES cycle augmented with the previous density, its last change and the
shipped warm-start network's predicted change, the second refinement sweep
with the previous step's second-sweep correction), extract velocities and
mu_eff, move the bodies, shear the lattice and rebuild the discretisation and
the proxy fit.  Beside it: iterations per step of the other starts (zero,
recycled directions without the network) and the plain FP64 solve (zero
start, double-precision pair sums) in seconds per shear time.

value: near-image pair evaluations (9 N^2 per operator application, every
FP32 and FP64 application counted) per second, whole job (all ranks), in
Gpairs/s.  Multi-GPU runs are independent replicas (weak scaling).

--impl reference times the FP64 CPU oracle (numpy) on a bounded sample of the
same workload and reports the same metric.
"""
import argparse
import hashlib
import json
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
WORKLOAD = "25 ellipses/cell, phi 0.3, AR U[1,3], gap>=1e-2, 256 nodes/body (N=6400), dt 1e-3"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--mixed-only", action="store_true",
                   help="time the mixed-precision steps only (no plain-FP64 comparison, no end-to-end loop); "
                        "used for kernel launch lists")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


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


def kernel_source(kernel):
    """Source text of a kernel in the library (from its name to the closing
    brace at column 0), the unit the committed ncu summaries are keyed on."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "paper_1912_04501_gb300", "csrc", "*.cu"))):
        text = open(path).read()
        k = text.find(kernel + "(")
        while k >= 0 and text.rfind("\n", 0, k) >= 0 and "__global__" not in text[text.rfind("__global__", 0, k):k][:400]:
            k = text.find(kernel + "(", k + 1)
        if k >= 0:
            e = text.find("\n}\n", k)
            return text[text.rfind("__global__", 0, k):e + 3]
    return ""


def source_hash(kernel):
    return hashlib.sha256(kernel_source(kernel).encode()).hexdigest()[:16]


def profiled_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the kernel's current source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_config2.md")
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
def oracle_sample(cell, target_seconds=15.0):
    """Time the FP64 oracle's operator at a sample of targets; returns
    (Gpairs/s, description, threads, seconds of the timed application)."""
    import numpy as np
    from oracle import bie as obie
    from oracle import geometry
    s = geometry.Suspension(cell["e1"], cell["e2"], cell["centre"], cell["mu"], cell["gamma"], cell["bodies"])
    sv = cell["solver"]
    op = obie.Operator(s, n_proxy=sv["n_proxy"], proxy_radius=sv["proxy_radius"], n_coll=sv["n_coll"])
    rng = np.random.default_rng(0)
    sigma = rng.standard_normal((s.N, 2))
    def timed(S):
        t0 = time.perf_counter()
        op.apply(sigma, targets=np.sort(rng.choice(s.N, S, replace=False)))
        return time.perf_counter() - t0
    t1, t2 = timed(32), timed(256)  # fixed cost + per-target cost
    per = max((t2 - t1) / 224, 1e-6)
    S = int(min(s.N, max(32, (target_seconds - max(t1 - 32 * per, 0.0)) / per)))
    idx = np.sort(rng.choice(s.N, S, replace=False))
    t0 = time.perf_counter()
    op.apply(sigma, targets=idx)
    dt = time.perf_counter() - t0
    pairs = 9.0 * S * s.N
    desc = (f"FP64 numpy oracle: one operator application evaluated at {S} of {s.N} targets "
            f"({pairs:.3g} near pairs + wall discrepancy + proxy fit), {dt:.1f} s")
    return pairs / dt / 1e9, desc, 1, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1912_04501_gb300 import workloads
    cell = workloads.config2()
    vals, secs = [], []
    desc = ""
    per = max(5.0, 120.0 / max(1, args.steps + args.warmup))
    for k in range(args.warmup + args.steps):
        v, desc, cores, dt = oracle_sample(cell, target_seconds=per)
        if k >= args.warmup:
            vals.append(v)
            secs.append(dt)
    v = statistics.mean(vals)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "step": "one oracle application at a bounded sample of the targets", "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
def whole_job(units, ms, dist, device):
    """Whole-job figures of independent replicas: the units of all ranks
    (sum) and the slowest rank's time (max).  dist None: one process."""
    if dist is None:
        return float(units), float(ms)
    import torch
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u[0]), float(t[0])


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

    cell = workloads.config2()
    dt = cell["dt"]
    N = sum(b["n"] for b in cell["bodies"])
    pairs_per_apply = 9.0 * N * N
    stream = torch.cuda.Stream()
    net = learn.default_net(device=local)
    mode = 2 if net is not None else 3
    # the default near-sum tile shape: fixed, so that a profiler run of this
    # command launches the same kernels as the timed one (the autotuner's
    # choice depends on timings, which a profiler distorts; on this cell it
    # differs from the default by ~2%); direct launches (replaying captured
    # graphs measured no faster here)
    ctx = bie.Context(cell, precision=bie.BIE_MIXED, device=local, warm_start=mode, autotune=0, graph=0)
    shape, _ = ctx.near_shape()
    near32 = "k_near32x2" if bie.NEAR32_SHAPES[shape][0] else "k_near32"
    ctx.set_stream(stream.cuda_stream)
    if net is not None:
        net.set_stream(stream.cuda_stream)
        ctx.set_warm_net(net)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    for _ in range(args.warmup):
        ctx.step(dt, 1)
    props = torch.cuda.get_device_properties(local)
    uuid = str(getattr(props, "uuid", "") or "")
    ctx.profile_read()
    ctx.profile(True)
    barrier()
    clocks = Clocks(uuid)
    total_ms = 0.0
    applies32 = applies64 = 0
    iters = []
    mu = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m, info = ctx.step(dt, 1)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        applies32 += info["applies32"]
        applies64 += info["applies64"]
        iters.append(info["iterations"])
        mu.append(float(m[0]))
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    prof = ctx.profile_read()
    ctx.profile(False)
    pairs = pairs_per_apply * (applies32 + applies64)  # applies64: FP64-class (double-float) residuals
    # whole job: units of all ranks / slowest rank's time
    pairs_all, t_ms = whole_job(pairs, total_ms, dist, "cuda")
    value = pairs_all / (t_ms / 1e3) / 1e9
    ms_per_step = t_ms / args.steps

    if args.mixed_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": ms_per_step, "mixed_only": True,
                              "gpu_launches": prof["launches"], "profile": prof}), flush=True)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return

    # iterations per step of the other starts on the same trajectory start
    starts = {}
    st0 = ctx.get_state()
    for m in (0, 3):
        cm = bie.Context(cell, precision=bie.BIE_MIXED, device=local, warm_start=m)
        cm.set_stream(stream.cuda_stream)
        cm.set_state(st0["t"], st0["e2"], st0["xc"], st0["theta"], st0["sigma"], st0["sigma_prev2"], st0["dt_prev"],
                     st0["d2"])
        its = [cm.step(dt, 1)[1]["iterations"] for _ in range(3)]
        starts[{0: "zero", 3: "recycled"}[m]] = statistics.mean(its)
        cm.close()
    starts["learned" if mode == 2 else "recycled (no network shipped)"] = statistics.mean(iters)

    # plain FP64 solve per step (zero start, double-precision pair sums)
    ctx64 = bie.Context(cell, precision=bie.BIE_FP64, device=local, warm_start=0)
    ctx64.set_stream(stream.cuda_stream)
    ctx64.step(dt, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n64 = 2
    _, info64 = ctx64.step(dt, n64)
    torch.cuda.synchronize()
    ms64 = (time.perf_counter() - t0) * 1e3 / n64
    ctx64.close()

    # end to end through the public API with host buffers
    st = ctx.get_state()
    host_in = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
               (("e2", st["e2"]), ("xc", st["xc"].ravel()), ("theta", st["theta"]), ("sigma", st["sigma"]),
                ("sigma_prev2", st["sigma_prev2"]), ("d2", st["d2"]))}
    e2e_steps = max(3, args.steps // 2)
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
    nb = len(cell["bodies"])
    h2d = (3 * nb + 2 + 3 * 2 * N) * 8   # centroids, angles, e2, density, previous density, sweep correction
    d2h = (8 * nb + 3 * 2 * N + 1) * 8  # body table, density, previous density, sweep correction, mu_eff

    pk, pk_src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s, FFMA = 2 flops
    fp64_peak = 1.25                                   # TFLOP/s, nominal GB300 FP64 (no measured figure)
    # plain FP64 solve uses native double near sums (k_near64)
    flops_per_pair = 18.0
    n32, n64, ndf = prof["near32_launches"], prof["near64_launches"], prof["neardf_launches"]
    ms32 = prof["near32_ms"] / max(1, n32)
    ms64_k = prof["near64_ms"] / max(1, n64)
    msdf = prof["neardf_ms"] / max(1, ndf)
    roof32 = {"kernel": near32, "bound": "alu", "unit": "TFLOP/s", "peak": fp32_peak,
              "achieved": flops_per_pair * pairs_per_apply / (ms32 / 1e3) / 1e12 if n32 else None,
              "launch_ms": ms32, "launches": n32, "device_ms_total": prof["near32_ms"],
              "peak_source": f"FP32 CUDA cores 152 SM x 128 lanes x 2 x {sm_max:.0f} MHz (sm_max_mhz of "
                             f"{pk_src} peaks file)",
              "traffic": profiled_traffic(near32)}
    roof64 = {"kernel": "k_near64", "bound": "alu", "unit": "TFLOP/s", "peak": fp64_peak,
              "achieved": flops_per_pair * pairs_per_apply / (ms64_k / 1e3) / 1e12 if n64 else None,
              "launch_ms": ms64_k, "launches": n64, "device_ms_total": prof["near64_ms"],
              "peak_source": "nominal GB300 FP64 rate (profiling recipe table), not measured",
              "traffic": profiled_traffic("k_near64")}
    # double-float pairs run on the FP32 pipe: measured against the FP32 peak,
    # counting the same 18 algorithmic flops per pair (the extra ~120 FP32
    # instructions per pair are the price of the 48-bit arithmetic)
    roofdf = {"kernel": "k_near_df", "bound": "alu", "unit": "TFLOP/s", "peak": fp32_peak,
              "achieved": flops_per_pair * pairs_per_apply / (msdf / 1e3) / 1e12 if ndf else None,
              "launch_ms": msdf, "launches": ndf, "device_ms_total": prof["neardf_ms"],
              "peak_source": roof32["peak_source"], "traffic": profiled_traffic("k_near_df")}
    for r in (roof32, roof64, roofdf):
        r["frac"] = r["achieved"] / r["peak"] if r["achieved"] else None
    ranked = sorted([roof32, roof64, roofdf], key=lambda r: -r["device_ms_total"])
    dom, other = ranked[0], [r for r in ranked[1:] if r["launches"]]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, cores, _ = oracle_sample(cell)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "bodies": nb,
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
                       "parallelism": f"{world} independent replica(s)"},
            "s_per_shear_time": ms_per_step / 1e3 / dt,
            "s_per_shear_time_fp64": ms64 / 1e3 / dt,
            # operator applications per second (all ranks), and the pairs of an
            # application outside the near sum: wall discrepancy (2m wall
            # points x the 6 far image rows/columns of every node, velocity
            # and traction) and proxy correction (every node x M proxies)
            "matvecs_per_s": world * (applies32 + applies64) / (t_ms / 1e3),
            "pairs_per_apply": {"near": pairs_per_apply,
                                "wall": 2.0 * cell["solver"]["n_coll"] * 6 * N,
                                "proxy": float(N * cell["solver"]["n_proxy"])},
            "solve": {"applies32": applies32, "applies64": applies64, "iterations_mean": statistics.mean(iters),
                      "mu_eff_last": mu[-1], "iterations_per_step_by_start": starts},
            "roofline": {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")},
            "roofline_detail": [dom] + other,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_pairs / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps},
            "gpu_launches": prof["launches"],
            "clocks": clk,
            "wall_s_timed": t_wall,
        }
        print(json.dumps(line), flush=True)
    ctx.set_warm_net(None)
    ctx.close()
    if net is not None:
        net.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
