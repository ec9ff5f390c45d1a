#!/usr/bin/env python3
"""SPH density + force throughput on GB300 (particle-updates per second).

One step is one kick-drift-kick step of the whole hot path through the C ABI
(`sph_step`): time-step reduction, half kick and drift, cell build (counting
sort, in-cell order), density loop with the smoothing-length solve, force
loop, second half kick.  Default workload: the 128^3 = 2,097,152-particle
jittered lattice in a periodic unit box (FP64 positions, FP32 pair math).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (under torchrun) every rank advances its own copy of the workload
(independent replicas: the configuration has no cross-rank exchange); value is
the whole-job rate.  `--impl reference` times the FP64 CPU oracle on bounded
samples of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH density+force particle-updates/s at 2M"
UNIT = "particle-updates/s"
# Flops per in-support pair of the oracle's formulas (every add, multiply,
# divide and square root counts 1; see the design notes for the tally):
# a Newton pass of the density loop (n_hat and dn_hat/dh only), the density
# loop's final pass at the converged h (every sum), and the force loop.
F_NEWTON = 33
F_DENSITY = 66
F_FORCE = 72
KERNELS = {"cubic": 0, "quartic": 1, "wendland_c2": 2}
# Starting viscosity parameter of the SPHENIX workloads (alpha_c starts at 0).
SPHENIX_ALPHA_V0 = 0.8


def launches_per_step(n_total: int, n_sims: int = 1, tree: bool = False, axis: bool = False,
                      sphenix: bool = False) -> int:
    """Kernel launches of one sph_step over n_total particles.

    Uniform grid: time-step reduction (3), kick/drift (1), cell build (8 + the
    radix sort: 1 + 5 per 8-bit digit of the cell id, whose range is
    8 n + 216 n_sims cells), two gathers (2), density (2), force (2), kick (1).
    Nested grids: the cell build without its sort (8), the tree build (two
    64-bit radix sorts of 30 + c and 34 + c bits, c the cell-id bits, plus
    key, source keys, levels, target keys, flags, a 3-kernel scan, groups,
    count, neighbour ranges: 12), the tree gather (1), density with the
    reverse-pair grouping (6), force gather (1), force (1).  Sorted
    interactions on the uniform grid add the per-cell axis orders (1).  The
    SPHENIX flavour adds the viscosity update (1), two gathers of its records
    (2) and the gradient pass (2)."""
    cap = 8 * n_total + 216 * n_sims
    cbits = 1
    while cbits < 30 and (1 << cbits) <= cap:
        cbits += 1
    radix = lambda bits: 1 + 5 * ((bits + 7) // 8)  # noqa: E731
    integrate = 3 + 1 + 1
    if not tree:
        return integrate + 8 + radix(cbits) + 2 + 2 + 2 + (1 if axis else 0) + (5 if sphenix else 0)
    return integrate + 8 + radix(30 + cbits) + radix(34 + cbits) + 12 + 1 + 6 + 1 + 1
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="lattice128")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--served-resident", type=float, default=0.25,
                    help="fraction of the live simulations' particles the device store holds")
    ap.add_argument("--served-seconds", type=float, default=6.0,
                    help="length of the served request trace at half the saturated rate")
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of oracle work for the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", choices=sorted(KERNELS), default="cubic",
                    help="latticeN / clusteredN: smoothing kernel")
    ap.add_argument("--hier", action="store_true",
                    help="latticeN: sub-steps of the time-step hierarchy (a smooth temperature profile)")
    ap.add_argument("--hier-levels", type=int, default=4,
                    help="--hier: bins 0..this (dt_max = 2^levels x the shortest CFL step)")
    ap.add_argument("--hier-options", default="",
                    help="--hier: comma-separated sub-step options: wakeup, predict, keep_cells; graph: "
                         "one sub-step captured in a CUDA graph and replayed")
    ap.add_argument("--hier-hot", type=float, default=0.0,
                    help="--hier: instead of the smooth profile, a hot sphere (u x 100) holding this "
                         "fraction of the particles in gas at u = 1: few particles on short steps")
    ap.add_argument("--active", type=float, default=0.0,
                    help="latticeN: time the loops on an active subset of this fraction (a "
                         "spherical region) against the full loops, instead of the step")
    ap.add_argument("--sphenix", action="store_true",
                    help="latticeN: the SPHENIX flavour (time-dependent viscosity, conduction)")
    ap.add_argument("--axis-sort", action="store_true",
                    help="uniform grid: sorted interactions in the density filter")
    ap.add_argument("--tune", action="store_true",
                    help="run the autotuner on the workload (latticeN, clusteredN, batchN) and print its "
                         "record: the chosen parameters, their time and the defaults' time")
    ap.add_argument("--lanes-per-target", type=int, default=0, choices=(0, 2, 4),
                    help="uniform grid: lanes per target of the loops (0: automatic)")
    ap.add_argument("--symmetric", action="store_true",
                    help="uniform grid: each force pair evaluated once (SPH_FLAG_SYMMETRIC)")
    ap.add_argument("--ref-budget", type=float, default=120.0,
                    help="seconds of oracle work for the whole --impl reference run")
    ap.add_argument("--no-batched", action="store_true",
                    help="lattice128 default line: skip the batched and served measurements")
    ap.add_argument("--batched-boxes", type=int, default=256)
    ap.add_argument("--batched-steps", type=int, default=10)
    ap.add_argument("--served-sims", type=int, default=200,
                    help="simulations of the served run inside the default line")
    return ap.parse_args()


def make_workload(name: str) -> dict:
    """latticeN: jittered N^3 lattice (uniform grid).  clusteredN / clusteredNM:
    N (or N million, binary: 2M = 2^21) particles in 64 Plummer spheres plus a
    30% uniform background (nested grids)."""
    from paper_2305_13380_gb300 import inputs
    if name.startswith("lattice"):
        n = int(name[len("lattice"):])
        p = inputs.lattice(n, seed=0)
        p["desc"] = (f"jittered lattice {n}^3 = {n ** 3} particles, periodic unit box, "
                     "jitter +-0.1 d, sigma_v = 0.01, u = 1 +- 1%, equal masses, seed 0")
        p["tree"] = False
        return p
    if name.startswith("clustered"):
        tail = name[len("clustered"):]
        n = int(tail[:-1]) << 20 if tail.endswith("M") else int(tail)
        p = inputs.clustered(n, n_spheres=64, seed=0)
        p["desc"] = (f"{n} particles: 70% in 64 Plummer spheres (scale radii log-uniform "
                     "0.002-0.02, centres uniform), 30% uniform background, periodic unit box, "
                     "u log-normal sigma 1, sigma_v = 0.05, seed 0; nested grids")
        p["tree"] = True
        return p
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------- clocks ---
class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [ln.strip().split(",") for ln in self.file.read().splitlines() if ln.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() in ("active", "1"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- oracle ----
def _f32(p):
    import numpy as np
    q = {k: p[k] for k in ("x", "y", "z", "L")}
    for k in ("vx", "vy", "vz", "m", "u", "h0"):
        q[k] = np.asarray(p[k], dtype=np.float32).astype(np.float64)
    return q


def oracle_sample(p, n_target: int, seed: int, sphenix: bool = False, kernel: int = 0):
    """Oracle density + force for the particles of a sub-cube holding about
    n_target particles (the density also runs on a margin of one support
    around it, which the force needs).  With sphenix, the SPHENIX evaluation:
    the viscosity update and the gradient pass on the margin too, then the
    SPHENIX force.  kernel: SPH_KERNEL_* of the run.  Returns (particles
    updated, seconds)."""
    import numpy as np

    import oracle
    q = _f32(p)
    L = q["L"]
    n = len(q["x"])
    side = L * min(1.0, (n_target / n) ** (1.0 / 3.0))
    rng = np.random.default_rng(seed)
    c0 = rng.uniform(0, L, 3)
    phys = oracle.Physics(kernel=kernel)
    gk = oracle.gamma_k(kernel)
    H = gk * float(np.max(q["h0"])) * 1.1

    def inside(s):
        d = [np.abs((q[k] - c0[i] + 0.5 * L) % L - 0.5 * L) for i, k in enumerate("xyz")]
        return np.where((d[0] < s / 2) & (d[1] < s / 2) & (d[2] < s / 2))[0]
    core = inside(side)
    if len(core):
        # the halo reaches one (generous) support of the core's particles;
        # wider particles outside it keep stand-in values from their h0
        H = gk * float(np.max(q["h0"][core])) * 1.5
    halo = inside(side + 2 * H)
    t0 = time.perf_counter()
    d = oracle.density(q, q["h0"], targets=halo, phys=phys)
    h0 = q["h0"]
    rho0 = q["m"] * (1.2348 / h0) ** 3
    P0 = (5.0 / 3.0 - 1.0) * q["u"] * rho0
    state = {"h": h0.copy(), "rho": rho0, "f": np.ones(n), "P": P0,
             "c": np.sqrt(5.0 / 3.0 * P0 / rho0), "B": np.full(n, 0.5)}
    for k in state:
        state[k][halo] = d[k]
    if not sphenix:
        oracle.force(q, state, targets=core, phys=phys)
        return len(core), time.perf_counter() - t0
    X = oracle.Sphenix()
    av = np.full(n, SPHENIX_ALPHA_V0)
    div = np.zeros(n)
    div[halo] = d["div_v"]
    dt = 1e-4 * float(np.min(q["h0"]))
    av = oracle.sphenix_alpha_v(dt, state["h"], state["c"], div, np.zeros(n), 2.0 * state["c"], av, X, phys)
    g = oracle.sphenix_gradient(q, state, av, np.zeros(n), dt, halo, X, phys)
    ac = np.zeros(n)
    ac[halo] = g["alpha_c"]
    oracle.sphenix_force(q, state, av, ac, targets=core, phys=phys)
    return len(core), time.perf_counter() - t0


def cpu_baseline(p, budget_s: float, sphenix: bool = False, kernel: int = 0) -> dict:
    import oracle
    oracle.build()
    # calibrate on a small sample, then size the timed sample to the budget
    n0, t0 = oracle_sample(p, 2000, seed=1, sphenix=sphenix, kernel=kernel)
    n_target = int(max(2000, min(len(p["x"]), n0 * budget_s / max(t0, 1e-3))))
    nu, sec = oracle_sample(p, n_target, seed=2, sphenix=sphenix, kernel=kernel)
    what = "SPHENIX density, viscosity update, gradient pass and force" if sphenix else "density + force"
    return {"value": nu / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{what}: {nu} particles of a sub-cube (density also on a one-support halo, "
                       f"grid build over all {len(p['x'])} particles included), "
                       f"{sec:.1f} s on 1 host core")}


def measured_hbm_gbs():
    """The measured copy bandwidth of this machine's GPUs (GB/s), if recorded."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # the earlier single GB300 measurement


def fof_workload(name: str):
    """fofN / fofNM: the clustered recipe with N (or N million, binary)
    particles and the linking length 0.2 of the mean spacing (Sec. 7.1)."""
    tail = name[len("fof"):] or "2M"
    n = int(tail[:-1]) << 20 if tail.endswith("M") else int(tail)
    p = make_workload(f"clustered{n}")
    p["link"] = 0.2 * float(p["L"]) * n ** (-1.0 / 3.0)
    p["desc"] = p["desc"].replace("; nested grids", "") + "; linking length 0.2 of the mean spacing"
    return p


def oracle_fof_sample(p, n_target: int, seed: int):
    """Oracle friends-of-friends on the particles of a sub-cube holding about
    n_target particles (same positions, box and linking length).  Returns
    (particles labelled, seconds)."""
    import numpy as np

    import oracle
    L, n = float(p["L"]), len(p["x"])
    side = L * min(1.0, (n_target / n) ** (1.0 / 3.0))
    c0 = np.random.default_rng(seed).uniform(0, L, 3)
    d = [np.abs((np.asarray(p[k]) - c0[i] + 0.5 * L) % L - 0.5 * L) for i, k in enumerate("xyz")]
    sel = np.where((d[0] < side / 2) & (d[1] < side / 2) & (d[2] < side / 2))[0]
    xs = [np.ascontiguousarray(np.asarray(p[k], dtype=np.float64)[sel]) for k in "xyz"]
    t0 = time.perf_counter()
    oracle.fof(*xs, L, p["link"])
    return len(sel), time.perf_counter() - t0


def run_fof(args, world: int, rank: int, local: int):
    """Friends-of-friends groups of the clustered box (sph_fof): every step
    rebuilds the cells at the linking length and labels every particle."""
    import torch
    from paper_2305_13380_gb300 import build as B
    B.build()
    from paper_2305_13380_gb300 import replicas, sph

    p = fof_workload(args.workload)
    n, L, b = len(p["x"]), float(p["L"]), p["link"]
    xyz = [torch.as_tensor(p[k], dtype=torch.float64, device="cuda") for k in "xyz"]
    group = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx = sph.Context(sph.sph_default_params(box_size=L, flags=sph.SPH_FLAG_TIMING))
    for _ in range(args.warmup):
        sph.sph_fof(ctx, *xyz, b, group)
    torch.cuda.synchronize()
    if sph.sph_status(ctx):
        raise SystemExit("device status set by the warm-up")
    kt0 = sph.sph_kernel_times(ctx)  # reset
    del kt0
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(None)
    time.sleep(0.25)
    replicas.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        sph.sph_fof(ctx, *xyz, b, group)
    e1.record(stream)
    torch.cuda.synchronize()
    replicas.barrier()
    clk = clocks.stop()
    kt = sph.sph_kernel_times(ctx)
    value, ms = replicas.job_throughput(n * args.steps, e0.elapsed_time(e1))
    g = group.cpu().numpy()
    import numpy as np
    _, counts = np.unique(g, return_counts=True)
    # end to end: positions in from pinned host memory, labels out, every step
    host_x = [t.cpu().pin_memory() for t in xyz]
    host_g = torch.empty(n, dtype=torch.int32).pin_memory()
    for it in range(2 + args.e2e_steps):
        if it == 2:
            torch.cuda.synchronize()
            e0.record(stream)
        for d, h in zip(xyz, host_x):
            d.copy_(h, non_blocking=True)
        sph.sph_fof(ctx, *xyz, b, group)
        host_g.copy_(group, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value, _ = replicas.job_throughput(n * args.e2e_steps, e0.elapsed_time(e1))
    # memory-bound kernels: algorithmic bytes of one call per particle: x, y,
    # z read (24), the sorted copy written and read back (16 + 16), the cell
    # key and slot (8), the labels initialised, read and written (12)
    fof_ms = kt["density"][0] / max(kt["density"][1], 1)
    bytes_call = n * (24 + 32 + 8 + 12)
    hbm = measured_hbm_gbs()
    roofline = {"bound": "hbm", "kernel": "k_fof_prep + k_fof_link + k_fof_label",
                "achieved": bytes_call / (fof_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": bytes_call / (fof_ms / 1e3) / 1e9 / hbm if hbm else None, "traffic": None,
                "bytes_per_launch": bytes_call}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        n0, t0 = oracle_fof_sample(p, 20000, seed=1)
        n_target = int(max(20000, min(n, n0 * args.cpu_budget / max(t0, 1e-3))))
        nu, sec = oracle_fof_sample(p, n_target, seed=2)
        cpu = {"value": nu / sec, "unit": "particles/s", "cores": 1, "kind": "oracle",
               "sample": f"{nu} particles of a sub-cube, {sec:.1f} s on 1 host core"}
    line = {
        "metric": "friends-of-friends particles/s (clustered, 2M)", "value": value,
        "unit": "particles/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": p["desc"], "particles": n, "link": b,
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "particles/s", "h2d_bytes_per_step": 24 * n,
                "d2h_bytes_per_step": 4 * n, "steps": args.e2e_steps},
        "gpu_launches": (launches_per_step(n, 1, False) - 12 + 3) * args.steps,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                   "reasons": clk["reasons"], "samples": clk["samples"]},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "breakdown_ms_per_step": {k: v[0] / args.steps for k, v in kt.items() if v[1]},
        "groups": int(len(counts)), "largest_group": int(counts.max()),
        "particles_in_groups_of_32_or_more": int(counts[counts >= 32].sum()),
        "device_status": sph.sph_status(ctx),
    }
    if rank == 0:
        print(json.dumps(line))


def run_reference(args, world: int, rank: int):
    if rank != 0:
        return
    import oracle
    oracle.build()
    fof = args.workload.startswith("fof")
    p = fof_workload(args.workload) if fof else make_workload(args.workload)
    metric, unit = (("friends-of-friends particles/s (clustered, 2M)", "particles/s") if fof
                    else (METRIC, UNIT))
    sample = ((lambda q, k, seed: oracle_fof_sample(q, k, seed)) if fof else
              (lambda q, k, seed: oracle_sample(q, k, seed, sphenix=args.sphenix,
                                                kernel=KERNELS[args.kernel])))
    # size every sample so that the whole run stays near args.ref_budget seconds
    n0, t0 = sample(p, 1000, seed=99)
    per_step = args.ref_budget / max(1, args.steps + args.warmup)
    n_target = int(max(200, min(len(p["x"]), n0 * per_step / max(t0, 1e-3))))
    for w in range(args.warmup):
        sample(p, n_target, seed=100 + w)
    done, sec = 0, 0.0
    for k in range(args.steps):
        nu, s = sample(p, n_target, seed=1000 + k)
        done += nu
        sec += s
    value = done / sec
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "desc": p["desc"],
                       "sample": f"{n_target}-particle sub-cubes per step"},
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} sub-cubes of ~{n_target} particles"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ ours ---
def _traffic(kernel: str, source: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source file of that kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2305_13380_gb300", "csrc", source + ".cu")
    try:
        rec = json.load(open(path))[kernel]
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("source_sha256") == sha:
            return rec["bytes_per_launch"]
    except (OSError, KeyError, ValueError):
        pass
    return None


def batch_measure(n_boxes: int, steps: int, warmup: int, plain_steps: int) -> dict:
    """The batched workload: n_boxes independent periodic boxes (N log-uniform
    in [1e3, 1e5], even boxes jittered lattices, odd ones Plummer-clustered),
    one sph_step per step for all boxes, captured in a CUDA graph, cell
    geometry from the autotuner; against the same boxes each stepped by its
    own sph_step call (one simulation per launch).  Per-step latencies from
    CUDA events on the pool's stream; the slowest rank's under replicas."""
    import numpy as np
    import torch

    from paper_2305_13380_gb300 import build as B
    B.build()
    from paper_2305_13380_gb300 import inputs, pool, replicas, sph, tune

    boxes = inputs.batch(n_boxes, seed0=0)
    n = sum(len(b["x"]) for b in boxes)
    t_tune = time.perf_counter()
    # the boxes split by the spread of their smoothing lengths (lattices may
    # take the uniform grid, clustered boxes need nested grids), each part
    # with its own tuned cell geometry; one pool per part, stepped together
    parts = tune.best_split(boxes, key=f"batch{n_boxes}")
    tune_s = time.perf_counter() - t_tune
    over_of = {}
    for idx, over in parts:
        for i in idx:
            over_of[i] = over
    prm = lambda i: sph.sph_default_params(**over_of[i])  # noqa: E731
    P = pool.Group([pool.Pool([boxes[i] for i in idx], sph.sph_default_params(**over)) for idx, over in parts])
    P.start()
    P.capture()
    for _ in range(warmup):
        P.replay()
    P.stream.synchronize()
    if P.status():
        raise SystemExit(f"device status {P.status()} after the batched warm-up")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    clocks = Clocks(None)
    time.sleep(0.25)
    replicas.barrier()
    ev[0].record(P.stream)
    for k in range(steps):
        P.replay()
        ev[k + 1].record(P.stream)
    P.stream.synchronize()
    replicas.barrier()
    clk = clocks.stop()
    per = np.array([ev[k].elapsed_time(ev[k + 1]) for k in range(steps)])
    p50 = replicas.max_over_ranks(float(np.percentile(per, 50)))
    p99 = replicas.max_over_ranks(float(np.percentile(per, 99)))
    rate, mean_ms = replicas.job_throughput(n, float(np.mean(per)))
    st = P.status()
    # one simulation per launch: every box has its own pool and context
    singles = [pool.Pool([b], prm(i), stream=P.stream) for i, b in enumerate(boxes)]
    for S in singles:
        S.start()
    for S in singles:
        S.step()
    P.stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(P.stream)
    for _ in range(plain_steps):
        for S in singles:
            S.step()
    e1.record(P.stream)
    P.stream.synchronize()
    plain_ms = replicas.max_over_ranks(e0.elapsed_time(e1) / plain_steps)
    return {"boxes": n_boxes, "particles": n, "steps": steps, "warmup": warmup,
            "p50_ms": p50, "p99_ms": p99, "mean_ms": mean_ms, "updates_per_s": rate,
            "plain_per_launch_ms": plain_ms, "plain_updates_per_s": replicas.sum_over_ranks(n) / (plain_ms / 1e3),
            "plain_steps": plain_steps, "speedup_vs_plain": plain_ms / mean_ms,
            "tuned": [{"boxes": len(idx), "particles": sum(len(boxes[i]["x"]) for i in idx), "params": over}
                      for idx, over in parts],
            "tune_s": tune_s,
            "gpu_launches": sum(launches_per_step(sum(len(boxes[i]["x"]) for i in idx), len(idx),
                                                  bool(over.get("flags", 0) & sph.SPH_FLAG_TREE))
                                for idx, over in parts) * steps,
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                       "reasons": clk["reasons"], "samples": clk["samples"]},
            "device_status": st}


def run_tune(args, world: int, rank: int, local: int):
    """The autotuner on one workload: every candidate timed over a few pool
    steps (CUDA events), the fastest kept; prints the record."""
    from paper_2305_13380_gb300 import build as B
    B.build()
    from paper_2305_13380_gb300 import inputs, tune
    if args.workload.startswith("batch"):
        # each part of the split (tune.partition) tuned on its own
        n_boxes = int(args.workload[len("batch"):] or 256)
        sims = inputs.batch(n_boxes, seed0=0)
        t0 = time.perf_counter()
        recs = []
        for k, idx in enumerate(tune.partition(sims)):
            part = [sims[i] for i in idx]
            rec = tune.tune(part, key=f"batch{n_boxes}|part{k}-{len(idx)}", steps=max(3, min(args.steps, 10)))
            recs.append({"boxes": len(idx), "particles": sum(len(s["x"]) for s in part), "best": rec["best"],
                         "best_ms": rec["best_ms"], "default_ms": rec["default_ms"], "candidates": rec["times"]})
        line = {"metric": "autotuned step time per part", "value": sum(r["best_ms"] for r in recs), "unit": "ms",
                "higher_is_better": False, "n_gpus": world,
                "config": {"workload": args.workload, "particles": sum(len(s["x"]) for s in sims)},
                "parts": recs, "tune_s": time.perf_counter() - t0}
        if rank == 0:
            print(json.dumps(line))
        return
    else:
        p = make_workload(args.workload)
        sims = [{k: v for k, v in p.items() if k not in ("desc", "tree")}]
        key = args.workload
    t0 = time.perf_counter()
    rec = tune.tune(sims, key=key, steps=max(3, min(args.steps, 10)))
    line = {"metric": "autotuned step time", "value": rec["best_ms"], "unit": "ms", "higher_is_better": False,
            "n_gpus": world, "config": {"workload": args.workload, "particles": sum(len(s["x"]) for s in sims)},
            "best": rec["best"], "default_ms": rec["default_ms"],
            "gain_vs_default": (rec["default_ms"] / rec["best_ms"]) if rec["default_ms"] else None,
            "candidates": rec["times"], "tune_s": time.perf_counter() - t0}
    if rank == 0:
        print(json.dumps(line))


def run_batch(args, world: int, rank: int, local: int):
    """256 independent boxes (config of the batched workload), printed as their
    own line (p50 latency as the value)."""
    n_boxes = int(args.workload[len("batch"):] or 256)
    b = batch_measure(n_boxes, args.steps, args.warmup, plain_steps=args.steps)
    line = {
        "metric": f"batched SPH step p50/p99 latency ({n_boxes} boxes)", "value": b["p50_ms"],
        "unit": "ms", "higher_is_better": False, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "boxes": n_boxes, "particles": b["particles"],
                   "desc": "periodic unit boxes, N log-uniform in [1e3, 1e5], even: jittered "
                           "lattice, odd: 4 Plummer spheres + background",
                   "tuned": b["tuned"]},
        "p50_ms": b["p50_ms"], "p99_ms": b["p99_ms"],
        "particle_updates_per_s": b["updates_per_s"],
        "plain_ms_per_step": b["plain_per_launch_ms"], "plain_particle_updates_per_s": b["plain_updates_per_s"],
        "speedup_vs_plain": b["speedup_vs_plain"],
        "gpu_launches": b["gpu_launches"], "clocks": b["clocks"], "device_status": b["device_status"]}
    if rank == 0:
        print(json.dumps(line))


def served_measure(n_sims: int, seconds: float, resident: float) -> dict:
    """Served workload: live simulations of two colliding spheres (radii
    0.1-0.3, 10^3-5x10^5 particles log-uniform, relative speed 0.5-2); the
    device store holds the fraction `resident` of their particles (an HBM
    budget below the all-resident footprint), the rest wait in pinned host
    memory and are admitted on request; step requests arrive as a Poisson
    process and are served with continuous batching (several batches in flight
    on their own streams).  Measured: the saturated rate of both paths (every
    request present at once), a trace at half the batched path's saturated rate
    (batched only: one simulation per launch cannot sustain it), and a trace at
    half the plain path's saturated rate, which both sustain, served both ways."""
    import numpy as np
    import torch

    from paper_2305_13380_gb300 import build as B
    B.build()
    from paper_2305_13380_gb300 import inputs, replicas, serve, sph, tune

    t_gen = time.perf_counter()
    sims = {s: inputs.two_spheres(seed=s) for s in range(n_sims)}
    gen_s = time.perf_counter() - t_gen
    total = sum(len(p["x"]) for p in sims.values())
    largest = max(len(p["x"]) for p in sims.values())
    slots = 3
    batch_cap = max(4 * largest, 4 << 20)
    store_n = max(int(resident * total), 2 * largest)
    budget = store_n * serve.STATE_BYTES + slots * batch_cap * (serve.STATE_BYTES + serve.SCRATCH_BYTES)
    # grid mode, margin and leaf size tuned on every 64th simulation
    sample = [sims[s] for s in range(0, n_sims, 64)]
    over = tune.best_params(sample, key=f"served-sample-{n_sims}")
    prm = sph.sph_default_params(**over)
    srv = serve.Server(budget, store_particles=store_n, slots=slots, batch_particles=batch_cap,
                       params=prm)
    for s, p in sims.items():
        srv.register(s, p)
    del sims
    ids = list(srv.sims)

    def reset():
        srv.finished, srv.n_batches, srv.updates, srv.batch_log = [], 0, 0, []

    def plain_mode(on: bool, keep=[]):
        # one simulation per launch on one stream, or continuous batching
        if on:
            keep[:] = [srv.slots, srv.max_batch_sims]
            srv.slots, srv.max_batch_sims = srv.slots[:1], 1
        else:
            srv.slots, srv.max_batch_sims = keep

    srv.run(serve.poisson_trace(6 * slots, rate=1e9, sims=ids, seed=0))   # warm-up
    reset()
    sat = srv.run(serve.poisson_trace(3 * slots * 32, rate=1e9, sims=ids, seed=1))
    cap_rate = sat["requests"] / sat["wall_s"]
    plain_mode(True)
    reset()
    psat = srv.run(serve.poisson_trace(96, rate=1e9, sims=ids, seed=3))
    plain_mode(False)
    plain_cap = psat["requests"] / psat["wall_s"]
    rate = 0.5 * cap_rate
    trace = serve.poisson_trace(max(200, int(rate * seconds)), rate=rate, sims=ids, seed=2)
    reset()
    up0, ev0 = srv.uploads, srv.evictions
    clocks = Clocks(None)
    time.sleep(0.25)
    replicas.barrier()
    out = srv.run(trace)
    replicas.barrier()
    clk = clocks.stop()
    paging = {"uploads": srv.uploads - up0, "evictions": srv.evictions - ev0}
    # like for like: a trace that both paths sustain, served both ways
    low = 0.5 * plain_cap
    ltrace = serve.poisson_trace(max(100, int(low * seconds)), rate=low, sims=ids, seed=4)
    reset()
    both_b = srv.run(ltrace)
    plain_mode(True)
    reset()
    both_p = srv.run(ltrace)
    plain_mode(False)
    req_rate, _ = replicas.job_throughput(out["requests"], 1e3 * out["wall_s"])
    pick = lambda r: {"p50_ms": replicas.max_over_ranks(r["p50_ms"]),  # noqa: E731
                      "p99_ms": replicas.max_over_ranks(r["p99_ms"]),
                      "particle_updates_per_s": replicas.sum_over_ranks(r["particle_updates_per_s"]),
                      "requests": r["requests"]}
    return {"simulations": n_sims, "particles": total, "resident_particles": store_n,
            "resident_fraction": store_n / total, "budget_gb": budget / 1e9, "slots": slots,
            "batch_particles": batch_cap, "generation_s": gen_s, "tuned": over,
            "saturated_requests_per_s": cap_rate, "plain_saturated_requests_per_s": plain_cap,
            "rate_per_s": rate, "p50_ms": replicas.max_over_ranks(out["p50_ms"]),
            "p99_ms": replicas.max_over_ranks(out["p99_ms"]), "mean_ms": out["mean_ms"],
            "requests": out["requests"], "requests_per_s": req_rate,
            "particle_updates_per_s": replicas.sum_over_ranks(out["particle_updates_per_s"]),
            "mean_sims_per_batch": out["mean_sims_per_batch"], "paging": paging,
            "batches": {k: out[k] for k in ("batches", "batch_sims_mean", "batch_particles_mean",
                                             "batch_ms_mean", "batch_ms_max")},
            "both_sustain": {"rate_per_s": low, "batched": pick(both_b), "plain": pick(both_p)},
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                       "reasons": clk["reasons"], "samples": clk["samples"]},
            "device_status": out["device_status"] | both_b["device_status"] | both_p["device_status"]}


def run_served(args, world: int, rank: int, local: int):
    """The served workload printed as its own line (p50 latency as the value)."""
    n_sims = int(args.workload[len("served"):] or 1000)
    r = served_measure(n_sims, args.served_seconds, args.served_resident)
    line = {
        "metric": f"served SPH step latency p50/p99 ({n_sims} live simulations)",
        "value": r["p50_ms"], "unit": "ms", "higher_is_better": False, "n_gpus": world,
        "steps": r["requests"], "warmup": 18, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "simulations": n_sims, "particles_resident": r["particles"],
                   "desc": "two uniform spheres per simulation, radii 0.1-0.3, N log-uniform in "
                           "[1e3, 5e5], relative speed 0.5-2, box 2; Poisson step requests",
                   "rate_per_s": r["rate_per_s"], "slots": r["slots"], "batch_particles": r["batch_particles"],
                   "resident_particles": r["resident_particles"], "resident_fraction": r["resident_fraction"],
                   "budget_gb": r["budget_gb"], "generation_s": r["generation_s"], "tuned": r["tuned"]},
        **{k: r[k] for k in ("p50_ms", "p99_ms", "mean_ms", "requests_per_s", "particle_updates_per_s",
                             "mean_sims_per_batch", "paging", "saturated_requests_per_s",
                             "plain_saturated_requests_per_s", "batches", "both_sustain", "clocks",
                             "device_status")},
    }
    if rank == 0:
        print(json.dumps(line))


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if args.tune:
        run_tune(args, world, rank, local)
    elif args.workload.startswith("batch"):
        run_batch(args, world, rank, local)
    elif args.workload.startswith("fof"):
        run_fof(args, world, rank, local)
    elif args.workload.startswith("served"):
        run_served(args, world, rank, local)
    elif args.hier:
        run_hier(args, world, rank, local)
    elif args.active > 0.0:
        run_active(args, world, rank, local)
    else:
        run_step(args, world, rank, local)
    if world > 1:
        dist.destroy_process_group()


def run_hier(args, world: int, rank: int, local: int):
    """Sub-steps of the time-step hierarchy with adaptive bins over
    args.hier_levels + 1 levels (dt_max = 2^levels times the shortest CFL
    step): on the lattice (uniform grid) with a smooth temperature profile,
    u = 10^sin(2 pi x / L) (sound speeds over a decade), or a hot sphere; on
    the clustered box (nested grids) with its own energies, where the small
    supports of the Plummer cores give the short steps."""
    import numpy as np
    import torch
    from paper_2305_13380_gb300 import build as B
    B.build()
    from paper_2305_13380_gb300 import replicas, sph

    p = make_workload(args.workload)
    tree = bool(p["tree"])
    n, L = len(p["x"]), float(p["L"])
    if tree:
        if args.hier_hot > 0.0:
            raise SystemExit("--hier-hot: lattice workloads only")
        profile = "the clustered box's log-normal u (Plummer cores: small h, short steps)"
    elif args.hier_hot > 0.0:
        # a hot sphere (sound speed x 10) in uniform gas: its particles step
        # 8-16 times shorter than the rest
        X = np.stack([np.asarray(p[k]) for k in ("x", "y", "z")], 1) - 0.5 * L
        r = np.sqrt((X ** 2).sum(1))
        rad = float(np.quantile(r, args.hier_hot))
        p["u"] = np.where(r <= rad, 100.0, 1.0)
        profile = f"hot sphere (u = 100) of {args.hier_hot:g} of the particles in u = 1"
    else:
        # a smooth temperature profile along x over a decade in sound speed:
        # hot and cold slabs with their own step lengths, no violent mixing
        p["u"] = 10.0 ** (np.sin(2.0 * np.pi * np.asarray(p["x"]) / L))
        profile = "10^sin(2 pi x / L)"
    t = sph.to_device(p)
    arrays = {k: t[k].clone() for k in ("x", "y", "z", "vx", "vy", "vz", "u", "m")}
    for k in ("h", "ax", "ay", "az", "du_dt", "v_sig", "rho", "f", "div_v", "curl_v", "P", "c", "balsara"):
        arrays[k] = torch.zeros(n, dtype=torch.float32, device="cuda")
    arrays["dt"] = torch.zeros(1, dtype=torch.float64, device="cuda")
    # nested grids: the tuner's choice for the clustered box (margin 0.03, 32
    # particles per leaf)
    gflags = sph.SPH_FLAG_TREE if tree else 0
    gprm = dict(cell_margin=0.03, n_leaf=32) if tree else {}
    init = sph.Context(sph.sph_default_params(box_size=L, flags=sph.SPH_FLAG_SYNC | gflags, **gprm))
    part = sph.particles(t)
    dout = sph.density_out({k: arrays[k] for k in sph.DENSITY_FIELDS})
    h_in = t["h0"]
    for _ in range(8):  # rebuild until the top cells hold every support
        cells = sph.sph_build_cells(init, t["x"], t["y"], t["z"], h_in)
        try:
            sph.sph_density(init, cells, part, h_in, dout)
            break
        except sph.SPHError as e:
            if e.code != sph.SPH_E_REBUILD:
                raise
            h_in = arrays["h"].clone()
    sph.sph_force(init, cells, part, dout, sph.force_out({k: arrays[k] for k in sph.FORCE_FIELDS}))
    max_bin = args.hier_levels
    dt_min = float((0.1 * 1.825742 * arrays["h"] / arrays["v_sig"]).min())
    dt_max = float(2 ** max_bin) * dt_min
    opts = {o: True for o in args.hier_options.split(",") if o}
    graph = opts.pop("graph", False)
    if set(opts) - {"wakeup", "predict", "keep_cells"}:
        raise SystemExit(f"unknown --hier-options {args.hier_options}")
    bins = torch.zeros(n, dtype=torch.int32, device="cuda")
    sph.sph_time_bins(init, cells, part, dout, arrays["v_sig"], 0.1, dt_max, max_bin, bins)
    init.close()
    # first half kicks of the starting steps
    half = (0.5 * dt_max) * torch.pow(2.0, -bins.double()).float()
    for k in ("x", "y", "z"):
        arrays["v" + k] += arrays["a" + k] * half
    arrays["u"] += arrays["du_dt"] * half
    pool = sph.pool(torch.tensor([0, n], dtype=torch.int64, device="cuda"),
                    torch.tensor([L], dtype=torch.float64, device="cuda"), arrays)
    tb = torch.zeros(n, dtype=torch.int64, device="cuda")
    # (the nested grids: a synchronous context, so that a support outgrowing
    # the top cells rebuilds and repeats the density inside the call)
    ctx = sph.Context(sph.sph_default_params(box_size=L, flags=sph.SPH_FLAG_TIMING | gflags |
                                             (sph.SPH_FLAG_SYNC if tree else 0), **gprm))
    tick = 0
    scratch = torch.zeros((), dtype=torch.int64, device="cuda")
    if graph:
        # one sub-step captured in a CUDA graph (the tick on the device), each
        # replay one more sub-step; launched from the context's stream
        if opts.get("keep_cells"):
            raise SystemExit("--hier-options graph: kept cells need the host (not capturable)")
        st = torch.cuda.Stream()
        ctx.close()
        ctx = sph.Context(sph.sph_default_params(box_size=L, flags=gflags, **gprm), st)
        tick_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
        with torch.cuda.stream(st):
            sph.sph_hier_substep_dev(ctx, pool, bins, tb, dt_max, max_bin, tick_dev, **opts)
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            sph.sph_hier_substep_dev(ctx, pool, bins, tb, dt_max, max_bin, tick_dev, **opts)
        for _ in range(args.warmup):
            with torch.cuda.stream(st):
                g.replay()
                scratch += (tb == tick_dev).sum()
        st.synchronize()
        tick = int(tick_dev.item())
    else:
        for _ in range(args.warmup):
            tick = sph.sph_hier_substep(ctx, pool, bins, tb, dt_max, max_bin, tick, **opts)
            scratch += (tb == tick).sum()  # loads the counting kernels before the timed region
    torch.cuda.synchronize()
    sph.sph_kernel_times(ctx)  # reset
    clocks = Clocks(None)
    replicas.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    active_dev = torch.zeros((), dtype=torch.int64, device="cuda")
    ticks0 = tick
    per_call = []
    if graph:
        with torch.cuda.stream(st):
            for _ in range(args.steps):
                c0 = time.perf_counter()
                g.replay()
                active_dev += (tb == tick_dev).sum()
                per_call.append(time.perf_counter() - c0)
        st.synchronize()
        tick = int(tick_dev.item())
    else:
        for _ in range(args.steps):
            c0 = time.perf_counter()
            tick = sph.sph_hier_substep(ctx, pool, bins, tb, dt_max, max_bin, tick, **opts)
            per_call.append(time.perf_counter() - c0)
            active_dev += (tb == tick).sum()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    active = int(active_dev.item())
    clk = clocks.stop()
    kt = sph.sph_kernel_times(ctx)
    if sph.sph_status(ctx):
        raise SystemExit("device status set in the hierarchy sub-steps")
    value, ms = replicas.job_throughput(active, wall * 1e3)
    levels = torch.bincount(bins.long(), minlength=max_bin + 1).tolist()
    line = {
        "metric": "SPH hierarchy sub-step active-particle updates/s",
        "value": value, "unit": "particle-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "particles": n, "max_bin": max_bin,
                   "u": profile, "bins_at_end": levels, "ticks": tick - ticks0,
                   "grid": "nested" if tree else "uniform",
                   "options": sorted(opts) + (["graph"] if graph else []), "cell_builds": kt["build"][1],
                   "mean_active_fraction": active / (args.steps * n),
                   "step": "sph_hier_substep (adaptive bins); host wall time, the call "
                           "waits for its tick"},
        "gpu_launches": None,
        "breakdown_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
        # (graph replays: the host's enqueue time only)
        "call_ms": {"median": 1e3 * float(np.median(per_call)), "max": 1e3 * float(np.max(per_call))},
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
    }
    if rank == 0:
        print(json.dumps(line))


def run_active(args, world: int, rank: int, local: int):
    """The density and force loops on an active subset (the particles of a
    spherical region holding the fraction args.active of the box), against the
    full loops on the same cells: what a step of the time-step hierarchy
    costs when only those particles' steps end."""
    import numpy as np
    import torch
    from paper_2305_13380_gb300 import build as B
    B.build()
    from paper_2305_13380_gb300 import replicas, sph

    p = make_workload(args.workload)
    if p["tree"]:
        raise SystemExit("the masked loops run on the uniform grid (latticeN workloads)")
    n, L = len(p["x"]), float(p["L"])
    c0 = np.full(3, 0.5 * L)
    d = [(np.asarray(p[k]) - c0[i] + 0.5 * L) % L - 0.5 * L for i, k in enumerate("xyz")]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    mask = r < np.quantile(r, args.active)
    n_act = int(mask.sum())
    t = sph.to_device(p)
    act = torch.tensor(mask.astype(np.uint8), device="cuda")
    ctx = sph.Context(sph.sph_default_params(box_size=L, flags=sph.SPH_FLAG_SYNC))
    part = sph.particles(t)
    dd, ff = sph.alloc_density(n), sph.alloc_force(n)
    cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], t["h0"])
    sph.sph_density(ctx, cells, part, t["h0"], sph.density_out(dd))
    sph.sph_force(ctx, cells, part, sph.density_out(dd), sph.force_out(ff))
    ctx.close()
    ctx = sph.Context(sph.sph_default_params(box_size=L, flags=sph.SPH_FLAG_TIMING))
    cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], dd["h"])
    dout, fout = sph.density_out(dd), sph.force_out(ff)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        replicas.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    def full():
        sph.sph_density(ctx, cells, part, dd["h"], dout)
        sph.sph_force(ctx, cells, part, dout, fout)

    def masked():
        sph.sph_density_active(ctx, cells, part, dd["h"], act, dout)
        sph.sph_force_active(ctx, cells, part, dout, act, fout)

    bins = torch.empty(n, dtype=torch.int32, device="cuda")

    def binning():  # CFL bins of every particle + the limiter's neighbour pass
        sph.sph_time_bins(ctx, cells, part, dout, ff["v_sig"], 0.1, 1.0, 30, bins)

    clocks = Clocks(None)
    sph.sph_kernel_times(ctx)  # reset
    ms_full = timed(full)
    kt_full = sph.sph_kernel_times(ctx)
    ms_act = timed(masked)
    kt_act = sph.sph_kernel_times(ctx)
    full()  # the bins follow a full force evaluation, whose density lists they reuse
    ms_bins = timed(binning)
    clk = clocks.stop()
    per = args.steps + args.warmup
    if sph.sph_status(ctx):
        raise SystemExit("device status set in the masked loops")
    value, ms = replicas.job_throughput(n_act, ms_act)
    line = {
        "metric": "SPH density+force active-particle updates/s (time-step hierarchy subset)",
        "value": value, "unit": "particle-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": p["desc"], "particles": n, "active": n_act,
                   "active_fraction": n_act / n, "subset": "a central sphere",
                   "step": "sph_density_active + sph_force_active on fixed cells"},
        "full_loops_ms": ms_full, "masked_over_full_time": ms_act / ms_full,
        "time_bins_ms": ms_bins,
        "breakdown_ms": {"full": {k: v[0] / per for k, v in kt_full.items()},
                         "masked": {k: v[0] / per for k, v in kt_act.items()}},
        "gpu_launches": 8 * args.steps,  # per iteration: two gathers + mask + loop + overflow loop, twice
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
    }
    if rank == 0:
        print(json.dumps(line))


def fp32_peak_tflops(reps: int = 5) -> float:
    """Measured FP32 fused-multiply-add rate of the current device (TFLOP/s):
    the best of `reps` timed launches of the FP32 probe, a benchmark-only
    shared object built beside the library (not part of it)."""
    import ctypes
    import torch
    from paper_2305_13380_gb300 import build as pkg_build
    probe = ctypes.CDLL(pkg_build.build_probe())
    probe.fp32_probe.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    probe.fp32_probe.restype = ctypes.c_int
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = sms * 8, 20000
    sink = torch.zeros(blocks, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    def launch():
        rc = probe.fp32_probe(blocks, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.c_void_p(st.cuda_stream))
        if rc != 0:
            raise RuntimeError(f"fp32_probe failed with {rc}")
    launch()
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        launch()
        e1.record(st)
        st.synchronize()
        flops = blocks * 256 * 8 * 2 * iters
        best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def run_step(args, world: int, rank: int, local: int):
    """The single-simulation workloads (latticeN, clusteredN): one sph_step
    of the whole box per step."""
    import torch
    from paper_2305_13380_gb300 import build as B
    B.build()
    from paper_2305_13380_gb300 import replicas, sph

    p = make_workload(args.workload)
    n = len(p["x"])
    L = float(p["L"])
    t = sph.to_device(p)
    dev = "cuda"
    # The state lives in one device buffer, in the order of the end-to-end
    # copies: the fields a step updates, then m, then the density outputs.
    # A caller that keeps its host copy in the same layout moves a step's
    # inputs and results with one copy each way.
    sphenix = bool(args.sphenix)
    kern = KERNELS[args.kernel]
    f64_keys = ("x", "y", "z")
    # SPHENIX carries alpha_V, alpha_c and the previous divergence from step
    # to step: they join the fields a step reads and updates
    carried = ("alpha_v", "alpha_c", "div_v") if sphenix else ()
    f32_keys = ("vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du_dt", "v_sig") + carried + ("m",) + \
        tuple(k for k in ("rho", "f", "div_v", "curl_v", "P", "c", "balsara") if k not in carried)
    offs, size = {}, 0
    for k in f64_keys + f32_keys:
        offs[k] = size
        size += -(-n * (8 if k in f64_keys else 4) // 256) * 256
    dbuf = torch.empty(max(size, 256), dtype=torch.uint8, device=dev)
    arrays = {}
    for k in f64_keys + f32_keys:
        wide = k in f64_keys
        arrays[k] = dbuf[offs[k]:offs[k] + n * (8 if wide else 4)].view(
            torch.float64 if wide else torch.float32)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u", "m"):
        arrays[k].copy_(t[k])
    arrays["dt"] = torch.zeros(1, dtype=torch.float64, device=dev)
    sim_offset = torch.tensor([0, n], dtype=torch.int64, device=dev)
    box = torch.tensor([L], dtype=torch.float64, device=dev)

    tree = sph.SPH_FLAG_TREE if p["tree"] else 0
    # grid-mode flags of every context of the run
    mode = tree | (sph.SPH_FLAG_AXIS_SORT if args.axis_sort and not tree else 0) | \
        (sph.SPH_FLAG_SYMMETRIC if args.symmetric and not tree else 0)
    knobs = {"lanes_per_target": args.lanes_per_target}
    tuned = None
    if args.workload in ("lattice128", "clustered2M") and not (args.axis_sort or args.symmetric or
                                                               args.lanes_per_target or sphenix or kern):
        # the default run takes the autotuner's choice for this workload (cached per GPU)
        from paper_2305_13380_gb300 import tune
        sims = [{k: v for k, v in p.items() if k not in ("desc", "tree")}]
        tuned = tune.best_params(sims, key=args.workload)
        knobs = {k: v for k, v in tuned.items() if k in ("cell_margin", "lanes_per_target", "n_leaf")}
        mode = (mode & ~(sph.SPH_FLAG_TREE | sph.SPH_FLAG_SYMMETRIC)) | (tuned.get("flags", 0) & (
            sph.SPH_FLAG_TREE | sph.SPH_FLAG_SYMMETRIC))
        tree = mode & sph.SPH_FLAG_TREE
    # initial density + force (untimed) through the single-simulation calls
    init = sph.Context(sph.sph_default_params(box_size=L, flags=sph.SPH_FLAG_SYNC | mode, kernel=kern, **knobs))
    part = sph.particles(t)
    dout = sph.density_out({k: arrays[k] for k in sph.DENSITY_FIELDS})
    h_in = t["h0"]
    for _ in range(8):
        cells = sph.sph_build_cells(init, t["x"], t["y"], t["z"], h_in)
        try:
            sph.sph_density(init, cells, part, h_in, dout)
            break
        except sph.SPHError as e:
            if e.code != sph.SPH_E_REBUILD:
                raise
            h_in = arrays["h"].clone()
    fout = sph.force_out({k: arrays[k] for k in sph.FORCE_FIELDS})
    X = sph.sph_sphenix_default_params()
    if sphenix:
        arrays["alpha_v"].fill_(SPHENIX_ALPHA_V0)
        arrays["alpha_c"].zero_()
        dvp = arrays["div_v"].clone()
        sph.sph_sphenix_gradient(init, cells, part, dout, X, 0.0,
                                 sph.sphenix_state(arrays["alpha_v"], arrays["alpha_c"], dvp, arrays["v_sig"]))
        sph.sph_force_sphenix(init, cells, part, dout, arrays["alpha_v"], arrays["alpha_c"], fout)
    else:
        sph.sph_force(init, cells, part, dout, fout)
    init.close()

    def step(c, pl):
        if sphenix:
            sph.sph_step_sphenix(c, pl, X, arrays["alpha_v"], arrays["alpha_c"])
        else:
            sph.sph_step(c, pl)

    ctx = sph.Context(sph.sph_default_params(box_size=L, flags=sph.SPH_FLAG_TIMING | mode, kernel=kern, **knobs))
    pool = sph.pool(sim_offset, box, arrays)
    for _ in range(args.warmup):
        step(ctx, pool)
    torch.cuda.synchronize()
    st = sph.sph_status(ctx)
    if st:
        raise SystemExit(f"device status {st} after warm-up")
    sph.sph_kernel_times(ctx)  # reset

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(gpu_id)
    time.sleep(0.25)
    replicas.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        step(ctx, pool)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    replicas.barrier()
    clk = clocks.stop()
    kt = sph.sph_kernel_times(ctx)
    st = sph.sph_status(ctx)
    # every rank advances its own copy: units of all ranks over the slowest time
    value, ms = replicas.job_throughput(n * args.steps, e0.elapsed_time(e1))

    # one more step (untimed) that counts pairs and Newton passes
    cnt = sph.Context(sph.sph_default_params(box_size=L, flags=sph.SPH_FLAG_COUNT_PAIRS | mode, kernel=kern, **knobs))
    arrays["n_iter"] = torch.zeros(n, dtype=torch.int32, device=dev)
    step(cnt, sph.pool(sim_offset, box, arrays))
    pairs_d, pairs_f = sph.sph_pair_counts(cnt)
    tree_counts = sph.sph_tree_counts(cnt) if tree else None
    mean_pass = float(arrays.pop("n_iter").double().mean().item())
    cnt.close()

    # end to end: the state in pinned host memory, in the device layout; every
    # step copies x .. v_sig (and the SPHENIX fields) and m in and the same
    # without m out.  A step's inputs are the previous step's results as the
    # host holds them: the read-back of step k and the upload of step k + 1
    # run in chunks on two streams, each chunk's upload after its own
    # read-back, so the two directions of the link overlap (every byte still
    # goes out and comes back through host memory)
    bi = offs["m"] + 4 * n          # x, y, z, v, u, h, a, du/dt, v_sig, [alpha_v, alpha_c, div_v,] m
    bo = offs["m"]                  # the same without m, which a step does not change
    host = torch.empty(bi, dtype=torch.uint8, pin_memory=True)
    host.copy_(dbuf[:bi])
    e2e_ctx = sph.Context(sph.sph_default_params(box_size=L, flags=mode, kernel=kern, **knobs))
    up = torch.cuda.Stream()
    n_chunk = 8
    cuts = [bo * c // n_chunk // 16 * 16 for c in range(n_chunk)] + [bo]
    ev = [torch.cuda.Event() for _ in range(n_chunk)]
    up_done = torch.cuda.Event()
    dbuf[:bi].copy_(host, non_blocking=True)
    # timed: from the read-back of step 1 to that of step 1 + e2e_steps (the
    # steps 2 .. 1 + e2e_steps with their uploads, and one read-back more)
    for it in range(2 + args.e2e_steps):
        if it > 0:
            stream.wait_event(up_done)   # this step's inputs are in
        step(e2e_ctx, pool)
        if it == 1:
            torch.cuda.synchronize()
            e0.record(stream)
        last = it == 1 + args.e2e_steps
        if not last:
            up.wait_stream(stream)
            with torch.cuda.stream(up):
                dbuf[bo:bi].copy_(host[bo:bi], non_blocking=True)   # m
        for c in range(n_chunk):
            host[cuts[c]:cuts[c + 1]].copy_(dbuf[cuts[c]:cuts[c + 1]], non_blocking=True)
            if not last:
                ev[c].record(stream)
                up.wait_event(ev[c])
                with torch.cuda.stream(up):
                    dbuf[cuts[c]:cuts[c + 1]].copy_(host[cuts[c]:cuts[c + 1]], non_blocking=True)
        if not last:
            up_done.record(up)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value, e2e_ms = replicas.job_throughput(n * args.e2e_steps, e0.elapsed_time(e1))
    if sph.sph_status(e2e_ctx):
        raise SystemExit("device status set in the end-to-end run")

    # roofline of each loop kernel (ALU bound: FP32 pipe, no tensor cores); the
    # line's "roofline" is the dominant one
    props = torch.cuda.get_device_properties(local)
    peak_mhz = clk["sm_max_mhz"] or 2070.0
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * peak_mhz * 1e6 / 1e12
    fma_peak = fp32_peak_tflops()  # measured FP32 FMA rate of this device
    loops = {}
    for kname, flops in (("density", pairs_d * (mean_pass * F_NEWTON + F_DENSITY)),
                         ("force", pairs_f * F_FORCE)):
        kms = kt[kname][0] / max(kt[kname][1], 1)
        achieved = flops / (kms / 1e3) / 1e12
        kfull = f"k_tree_{kname}" if tree else f"k_{kname}"
        loops[kfull] = {
            "bound": "alu", "kernel": kfull, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_measured_fma": fma_peak, "frac_of_measured": achieved / fma_peak,
            # the records hold the cubic-spline instances' counters
            "traffic": _traffic(kfull[2:], "tree_loops" if tree else kname) if kern == 0 else None,
            "peak_basis": (f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 "
                           f"lanes x 2 flop x {peak_mhz:.0f} MHz (derived; no measured FP32 "
                           "peak in MEASURED_PEAKS.json)"),
            "launch_ms": kms, "flops_per_launch": flops,
            "flops_basis": (f"{pairs_d} pairs x ({mean_pass:.4f} Newton passes x {F_NEWTON} + {F_DENSITY})"
                            if kname == "density" else f"{pairs_f} pairs x {F_FORCE}")}
    roofline = max(loops.values(), key=lambda r: r["launch_ms"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, args.cpu_budget, sphenix, kern)

    # the metric's second half: batched step latency (and a short served run)
    batched = served = None
    if (args.workload == "lattice128" and not args.no_batched and not sphenix and kern == 0
            and not args.axis_sort and not args.symmetric):
        ctx.close()
        e2e_ctx.close()
        del dbuf, arrays, pool, host
        torch.cuda.empty_cache()
        batched = batch_measure(args.batched_boxes, args.batched_steps, 3, plain_steps=2)
        torch.cuda.empty_cache()
        served = served_measure(args.served_sims, 3.0, args.served_resident)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": p["desc"], "particles_per_gpu": n,
                   "step": ("sph_step_sphenix: dt, kick+drift, cell build, density (h solve), viscosity "
                            "update, gradient pass (lap u, alpha_c), SPHENIX force, kick" if sphenix else
                            "sph_step: dt, kick+drift, cell build, density (h solve), force, kick"),
                   "flavour": "SPHENIX" if sphenix else "Minimal",
                   "kernel": args.kernel,
                   "l2": "inputs larger than L2: each step touches ~0.5 GB of state and scratch",
                   "parallelism": f"replicas x{world}",
                   "grid": ("nested grids" if tree else
                            "uniform, sorted interactions" if mode & sph.SPH_FLAG_AXIS_SORT else "uniform"),
                   "force_pairs": "each pair once (symmetric)" if mode & sph.SPH_FLAG_SYMMETRIC else "gather",
                   "params": {"cell_margin": knobs.get("cell_margin", 0.05),
                              "lanes_per_target": knobs.get("lanes_per_target", 0),
                              "tuned": tuned is not None}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo, "steps": args.e2e_steps},
        "gpu_launches": launches_per_step(n, 1, bool(tree), bool(mode & sph.SPH_FLAG_AXIS_SORT),
                                          sphenix) * args.steps,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                   "reasons": clk["reasons"], "samples": clk["samples"]},
        "roofline": roofline,
        "roofline_loops": loops,
        "cpu_baseline": cpu,
        "batched": batched,
        "served": served,
        "breakdown_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
        # the loops alone: density (all Newton passes) + force per step
        "density_force_updates_per_s": n / ((kt["density"][0] + kt["force"][0]) / args.steps / 1e3),
        "pairs_per_step": {"density_final_pass": pairs_d, "force": pairs_f,
                           "mean_newton_passes": mean_pass},
        "nested_grids": tree_counts,
        "device_status": st,
        "wall_s": wall,
    }
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
