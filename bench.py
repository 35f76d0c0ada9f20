"""Throughput benchmark of the fused two-component pseudopotential LBM step on GB300.

Workload (one GPU): the cylinder contact-angle case scaled to 1024x1024 (cylinder radius 160,
droplet radius 200), seven adhesion values lambda targeting theta = 30..150 degrees, FP32 compute
and FP32 SoA storage, run as one seven-case ensemble.  One bench step is one pass of the whole hot
path over that batch: 100 time steps (fused collide-stream-force kernel, one launch per time step,
replayed from a captured CUDA graph), then the FP64 diagnostics reduction and the contact-angle
measurement of every case.

Metric: MLUPS = lattice nodes x time steps / second over all nodes of all cases (whole job).
Timed region: W warm-up steps, then exactly K steps between a barrier + synchronize on both sides,
CUDA events on the library's stream; the populations (1.06 GB per buffer) are far larger than L2.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
                    [--workload sweep|throat|porous|ensemble] [--storage f32|f16|bf16|f64]

The other workloads measure the remaining configurations the same way (one JSON line each): the
2048x512 throat channel as 8 replicas (so that even 16-bit state exceeds L2), the 4096x2048 porous
medium with inlet and outflow, and the 256-case uneven ensemble plus the co-current channel.

Under torchrun each rank runs its own seven cases (weak scaling, no collective on the data path);
rank 0 prints the JSON line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS (2-comp D2Q9) & % of GB300 HBM peak; FP32/FP16-store vs FP64 at stated error"
UNIT = "MLUPS"
INNER = 100            # time steps per bench step
BYTES_PER_NODE = {"f32": 144, "f16": 72, "bf16": 72, "f64": 288}
KERNEL_SOURCES = ("paper_2505_22256_gb300/csrc/lbm_step.cu", "paper_2505_22256_gb300/csrc/lbm_device.cuh",
                  "paper_2505_22256_gb300/csrc/lbm_tma.cuh")
KERNEL_SOURCES_3D = ("paper_2505_22256_gb300/csrc/lbm3d.cu", "paper_2505_22256_gb300/csrc/lbm_device.cuh")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "f64"])
    ap.add_argument("--workload", default="sweep", choices=list(WORKLOADS),
                    help="sweep: 7 cylinder cases of 1024^2 (the headline); throat: 8 replicas of the "
                         "2048x512 throat channel; porous: 4096x2048 porous medium with inlet/outflow; "
                         "ensemble: 256 uneven cases + the 4096x256 co-current channel; compare: the "
                         "sweep under the improved and the original scheme (14 cases); obstacle: 64 "
                         "replicas of the 350x150 square-obstacle channel (Poiseuille inlet); couette: "
                         "512 replicas of the 50x100 two-layer Couette channel (sliding walls); sphere3d: "
                         "the 3-D droplet on a sphere, 200x200x280 (Sec. 3.5)")
    ap.add_argument("--n", type=int, default=1024, help="sweep: lattice side of each case")
    ap.add_argument("--size", default=None, help="throat / porous: lattice WxH (default 2048x512 / 4096x2048); "
                                                 "sphere3d: n for the geometry scaled to n x n x 1.4n")
    ap.add_argument("--cases", type=int, default=7, help="sweep: number of lambda values (1..7)")
    ap.add_argument("--inner", type=int, default=INNER, help="time steps per bench step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--wall-inline", type=int, default=None, choices=[0, 1],
                    help="with --no-autotune: the step kernel's wall-list form (1 inlined, 0 called)")
    ap.add_argument("--launch-table", action="store_true",
                    help="instead of the bench line: every launch shape the autotuner tries (wall-list "
                         "form x block width x row chunks), one untimed and three timed steps each, one "
                         "JSON line with the table (a capture of it under ncu gives the per-shape "
                         "counters in the same order)")
    ap.add_argument("--no-modes", action="store_true",
                    help="skip the FP16 storage form measured beside an FP32 line at one GPU")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--split", action="store_true",
                    help="strong scaling: every rank builds the same workload and steps only its share "
                         "of the cases, assigned by node count (longest first, to the least-loaded rank)")
    return ap.parse_args(argv)


WORKLOADS = ("sweep", "throat", "porous", "ensemble", "compare", "obstacle", "couette", "sphere3d")
BYTES_PER_NODE_3D = {"f32": 304, "f64": 608, "f16": 152, "bf16": 152}  # 2 components x 19 populations, read + written


# ------------------------------------------------------------------------------------------------
# Multi-rank plumbing (one process per GPU, no collective on the data path)
# ------------------------------------------------------------------------------------------------
def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of every rank's value (a job takes its slowest rank's time); the value itself
    when the job runs alone."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world: int, nodes_per_rank: int, steps_per_rank: int, total_ms: float) -> float:
    """Whole-job lattice updates per second (millions): every rank updates nodes_per_rank nodes
    steps_per_rank times (weak scaling) within the job's time total_ms.  Under --split the caller
    passes world = 1 and the nodes of the whole job."""
    return world * nodes_per_rank * steps_per_rank / (total_ms / 1e3) / 1e6


def lpt_shares(sizes, world: int) -> list:
    """Case indices per rank: cases in decreasing size (ties: lower index first), each to the rank
    with the least work so far (ties: lower rank).  Deterministic, so every rank computes the same
    partition from the same sizes without a collective.  The largest load is at most the mean load
    plus the largest case (the longest-processing-time rule)."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    shares = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        shares[r].append(i)
        load[r] += sizes[i]
    return [sorted(sh) for sh in shares]


def shard(cases, rank: int, world: int):
    """(this rank's cases, nodes of the whole job) under --split."""
    if world > len(cases):
        raise SystemExit(f"--split: {world} ranks for {len(cases)} cases")
    sizes = [c.nx * c.ny for c in cases]
    return [cases[i] for i in lpt_shares(sizes, world)[rank]], sum(sizes)


def workload(args, rank=0):
    """(cases, description) of the chosen workload; rank offsets the seeds (weak scaling)."""
    from paper_2505_22256_gb300 import scenarios as S

    if args.workload == "throat":
        nx, ny = map(int, (args.size or "2048x512").split("x"))
        k = ny / 512.0  # geometry scales with the channel height
        cases = [S.throat_channel(nx=nx, ny=ny, R=180.0 * k, r=120.0 * k, seed=3 + 100 * j + 1000 * rank)
                 for j in range(8)]
        return cases, (f"throat channel, 8 replicas of {nx}x{ny} per GPU (half-disks R={180 * k:g}, "
                       f"droplet r={120 * k:g}, g=1e-6, lambda for theta=90 deg)")
    if args.workload == "porous":
        nx, ny = map(int, (args.size or "4096x2048").split("x"))
        keep = max(8, 64 * nx // 4096)
        return [S.porous_disks(nx=nx, ny=ny, keep_out=(keep, keep), seed=4 + 1000 * rank)], \
            (f"porous medium {nx}x{ny} per GPU (disks r=12..40, porosity 0.6, inlet u=0.005 at x=0, outflow)")
    if args.workload == "ensemble":
        return S.ensemble_cases(256, seed=5 + 1000 * rank) + [S.cocurrent_channel(seed=6 + 1000 * rank)], \
            ("uneven ensemble per GPU: 256 square cases n=64..512 (flat wall / cylinder, lambda 0.22..2.17) "
             "+ the 4096x256 co-current channel")
    if args.workload == "obstacle":
        return [S.square_obstacle_channel(seed=8 + 100 * j + 1000 * rank) for j in range(64)], \
            ("square-obstacle microchannel, 64 replicas of 350x150 per GPU (Poiseuille inlet Re=7.5, outflow, "
             "square side 25, droplet r=25, theta 30.2 deg)")
    if args.workload == "couette":
        return [S.couette_channel(seed=7 + 100 * j + 1000 * rank) for j in range(512)], \
            "two-layer Couette flow, 512 replicas of 50x100 per GPU (walls sliding at -/+0.005)"
    angles = (30, 50, 70, 90, 110, 130, 150)[: args.cases]
    if args.workload == "compare":
        return S.scheme_comparison(n=args.n, seed=2 + 1000 * rank, angles=angles), \
            (f"scheme comparison, {len(angles)} cylinder cases of {args.n}x{args.n} per GPU under the improved "
             f"and the original scheme ({2 * len(angles)} cases)")
    return S.lambda_sweep_cylinder(n=args.n, seed=2 + 1000 * rank, angles=angles), \
        (f"cylinder contact-angle sweep, {len(angles)} cases of {args.n}x{args.n} per GPU "
         f"(R={160 * args.n // 1024}, r={200 * args.n // 1024}, lambda for theta=30..150 deg)")


def config_dict(args, cases, desc, world, split_nodes=None):
    nodes = sum(c.nx * c.ny for c in cases)
    fluid = sum(int((c.solid == 0).sum()) for c in cases)
    if split_nodes is None:
        par = {"parallelism": f"ensemble x{world} (no collective)"}
    else:  # the whole workload once, its cases shared out over the ranks
        desc = desc.replace(" per GPU", "")
        par = {"parallelism": f"cases split over {world} rank{'s' if world != 1 else ''} by node count "
                              "(no collective)",
               "job_nodes": split_nodes}
    return {
        "workload": f"{desc}, {args.inner} time steps + diagnostics + contact angle per step",
        "storage": args.storage, "cases_per_gpu": len(cases), "nodes_per_gpu": nodes,
        "fluid_nodes_per_gpu": fluid, "inner_steps": args.inner, **par,
        "l2": "inputs larger than L2 (state %.2f GB per buffer)" % (nodes * BYTES_PER_NODE[args.storage] / 2 / 1e9),
        **({"storage_shift_rho0": list(cases[0].rho0_store)} if args.storage in ("f16", "bf16") else {}),
    }


# ------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 6:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, p[2:6]):
                if v.lower() in ("active", "1"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# measured peaks and the committed ncu counters
# ------------------------------------------------------------------------------------------------
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for rel in sources:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


STORE_TYPE = {"f32": "float, float", "f16": "__half, float", "bf16": "__nv_bfloat16, float", "f64": "double, double"}


def step_kernel_name(storage: str, info: dict) -> str:
    """The step kernel's template instantiation as ncu names it (storage type, compute type, fields
    pass off, wall-list correction inlined or called, block width)."""
    return f"k_step<{STORE_TYPE[storage]}, 0, {info['wall_inline']}, {info['block_threads']}>"


def counter_records(path: str) -> list[dict]:
    """The records of a counter summary: `key: value` lines, `#` comments; a file may hold several
    records separated by `---` lines, each inheriting the keys above the first separator."""
    recs, cur = [], {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("---"):
                recs.append(cur)
                cur = {}
            elif ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                cur[k.strip()] = v.strip()
    recs.append(cur)
    return recs if len(recs) == 1 else [{**recs[0], **r} for r in recs[1:]]


def committed_traffic(storage: str, nodes_per_launch: int, prefix: str = "k_step", sources=KERNEL_SOURCES,
                      launch: dict | None = None):
    """DRAM bytes per launch from a committed ncu summary, scaled to this launch's nodes; None when
    no record was taken on this version of the kernel source or (launch given) on this
    instantiation and launch shape of the kernel.  The summaries are
    profiles/<prefix>_<storage>_counters.txt and profiles/<prefix>_<storage>_counters_<variant>.txt."""
    paths = [os.path.join(ROOT, "profiles", f"{prefix}_{storage}_counters.txt")]
    paths += sorted(glob.glob(os.path.join(ROOT, "profiles", f"{prefix}_{storage}_counters_*.txt")))
    for p in paths:
        try:
            recs = counter_records(p)
        except OSError:
            continue
        for kv in recs:
            try:
                if kv.get("kernel_source_sha256_16") != kernel_source_hash(sources):
                    continue
                if any(kv.get(key) != str(want) for key, want in (launch or {}).items()):
                    continue
                return float(kv["dram_bytes_per_launch"]) / float(kv["nodes_per_launch"]) * nodes_per_launch
            except (KeyError, ValueError):
                continue
    return None


# ------------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on a bounded sample of the same workload
# ------------------------------------------------------------------------------------------------
def host_info() -> dict:
    """The host cores the oracle runs on: their count and, where the system reports it, the model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu": model or platform.processor() or platform.machine()}


# max relative |d rho| after PARITY_STEPS steps that the GPU tests hold each storage mode to
PARITY_STEPS = 100
PARITY_BAR = {"f32": 1e-5, "f16": 5e-3, "bf16": 5e-2, "f64": 1e-10}


def parity_record(storage, case, err_rho, err_u, bar_note=None) -> dict:
    rec = {"storage": storage, "steps": PARITY_STEPS, "case": case, "max_rel_drho": err_rho, "max_abs_du": err_u,
           "bar_max_rel_drho": PARITY_BAR.get(storage), "within_bar": err_rho <= PARITY_BAR.get(storage, 0.0)}
    if bar_note:
        rec["bar_note"] = bar_note
    return rec


def cpu_baseline(args, seconds: float, parity: bool = False, also=()) -> dict:
    """The FP64 oracle timed on one case of the workload.  parity: also run that case on the GPU in
    the bench's storage mode (and in each storage mode of `also`) from the same initial state and
    report its error against the oracle's fields after PARITY_STEPS steps (the oracle's first
    PARITY_STEPS steps are part of the timed sample)."""
    import numpy as np

    import oracle

    cases, _ = workload(args)
    sc = max(cases, key=lambda c: c.nx * c.ny) if args.workload != "sweep" else cases[len(cases) // 2]
    cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
    f = oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0)
    need = PARITY_STEPS if parity else 1
    snap = None
    n = 0
    t0 = time.perf_counter()
    while True:
        f = oracle.run(cfg, sc.solid, f, 1)
        n += 1
        if parity and n == PARITY_STEPS:
            snap = f.copy()
        el = time.perf_counter() - t0
        if (el >= seconds and n >= need) or n >= 10000:
            break
    mlups = sc.nx * sc.ny * n / el / 1e6
    out = {"value": mlups, "unit": UNIT, "cores": cfg.nthreads, "kind": "oracle", "sample_s": el,
           "sample_updates": sc.nx * sc.ny * n,
           "sample": f"1 of the {len(cases)} cases ({sc.nx}x{sc.ny}, {sc.name}), {n} FP64 time steps "
                     f"in {el:.1f} s on {cfg.nthreads} host threads", "host": host_info()}
    if parity:
        # the same oracle on one host thread, continuing from the state reached (about 4 s)
        cfg1 = oracle.Config(nx=sc.nx, ny=sc.ny, nthreads=1, **sc.params())
        n1, t1 = 0, time.perf_counter()
        while True:
            f = oracle.run(cfg1, sc.solid, f, 1)
            n1 += 1
            el1 = time.perf_counter() - t1
            if el1 >= min(4.0, seconds) or n1 >= 10000:
                break
        out["single_thread_value"] = sc.nx * sc.ny * n1 / el1 / 1e6
        out["single_thread_sample"] = f"{n1} FP64 time steps of the same case in {el1:.1f} s on 1 host thread"
    if parity and snap is not None:
        from paper_2505_22256_gb300 import lbm

        o = oracle.fields(cfg, sc.solid, snap)
        fl = sc.solid == 0
        for st in (args.storage, *also):
            lat = lbm.Lattice(sc, st)
            lat.step(PARITY_STEPS)
            g = lat.fields()
            lat.close()
            err_rho = max(float(np.max(np.abs(g[k] - o[k])[fl] / o[k][fl])) for k in (0, 1))
            err_u = max(float(np.max(np.abs(g[k] - o[k])[fl])) for k in (2, 3))
            rec = parity_record(st, f"{sc.name} ({sc.nx}x{sc.ny})", err_rho, err_u)
            if st == args.storage:
                out["parity"] = rec
            else:
                out.setdefault("parity_storage_modes", {})[st] = rec
    return out


def extrapolation(full_updates: float, sample_updates: float, mlups: float) -> dict:
    """How the reference arm's rate relates to a full bench step: each timed step of that arm is a
    bounded sample (time steps of one case), so ms_per_step and steps are what ran, and the value, a
    rate, carries over to the full workload by this factor of updates."""
    return {"value_is_rate_of_sample": True, "sample_updates_per_step": int(sample_updates),
            "full_step_updates": int(full_updates), "factor": full_updates / sample_updates,
            "full_step_ms_at_this_rate": full_updates / (mlups * 1e6) * 1e3}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    if args.workload == "sphere3d":
        vals, secs, ups, base = [], [], [], None
        for k in range(args.warmup + args.steps):
            b = cpu_baseline_3d(per_step)
            if k >= args.warmup:
                vals.append(b["value"])
                secs.append(b["sample_s"])
                ups.append(b["sample_updates"])
                base = b
        value = statistics.mean(vals)
        nodes = 200 * 200 * 280
        line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": statistics.mean(secs) * 1e3, "higher_is_better": True, "scaling": "weak",
                "extrapolated": extrapolation(nodes * args.inner, statistics.mean(ups), value),
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "3-D droplet on a sphere, 200x200x280 per GPU (R=50, r=45, lambda=1, periodic)",
                           "storage": args.storage, "inner_steps": args.inner},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                                 "sample": base["sample"]},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    cases, desc = workload(args)
    split_nodes = None
    if args.split:  # describe rank 0's share, as our arm's rank 0 does
        cases, split_nodes = shard(cases, 0, args.gpus)
    # each step: a bounded sample of the workload (time steps of one case), sized so that the whole
    # --steps/--warmup run stays within a few minutes
    base = None
    vals, secs, ups = [], [], []
    for k in range(args.warmup + args.steps):
        b = cpu_baseline(args, per_step)
        if k >= args.warmup:
            vals.append(b["value"])
            secs.append(b["sample_s"])
            ups.append(b["sample_updates"])
            base = b
    value = statistics.mean(vals)
    full_updates = sum(c.nx * c.ny for c in cases) * args.inner
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(secs) * 1e3,
            "extrapolated": extrapolation(full_updates, statistics.mean(ups), value), "higher_is_better": True,
            "scaling": "strong" if args.split else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, cases, desc, args.gpus if args.split else 1, split_nodes),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
# the candidates of lbm_autotune: wall-list form, block width, row chunks (0 guided, < 0 guided with
# short tail items, > 0 uniform)
LAUNCH_SHAPES = [(w, t, r) for w in (0, 1) for t in (128, 64) for r in (0, -8, 16, 32, 64, 128)]


def launch_table(args, lat, stream) -> int:
    """Every launch shape the autotuner tries: one untimed and three single-launch steps each (under
    ncu, launch k of the capture belongs to shape k // 4 of the printed order), then, in a second
    pass, the mean time per launch over 16 steps in each shape.  Prints one JSON line."""
    import torch

    from paper_2505_22256_gb300 import lbm

    shapes, rows = [], []
    for w, t, r in LAUNCH_SHAPES:
        try:
            lbm.lbm_set_launch(lat.ctx, t, r)
        except lbm.LbmError:
            continue
        lbm.lbm_set_wall_path(lat.ctx, w)
        info = lat.info()
        for _ in range(4):
            lat.step(1)
        shapes.append((w, t, r))
        rows.append({"wall_inline": w, "block_threads": t, "rows_arg": r, "kernel": step_kernel_name(args.storage, info),
                     "block_rows": info["block_rows"], "grid_blocks": info["grid_blocks"],
                     "work_items": info["work_items"]})
    for (w, t, r), row in zip(shapes, rows):
        lbm.lbm_set_launch(lat.ctx, t, r)
        lbm.lbm_set_wall_path(lat.ctx, w)
        lat.step(2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(16)
        e1.record(stream)
        e1.synchronize()
        row["ms_per_launch"] = e0.elapsed_time(e1) / 16
    lat.close()
    print(json.dumps({"launch_table": rows, "storage": args.storage, "workload": args.workload}))
    return 0


def storage_mode_line(args, cases, storage: str, stream) -> dict:
    """The same workload in another storage mode, on the same GPU: the library's autotuner, then
    MODE_STEPS bench steps (time steps only) timed with CUDA events on the library's stream, after
    two untimed ones."""
    import torch

    from paper_2505_22256_gb300 import lbm

    lat = lbm.Lattice(cases, storage=storage, cuda_stream=stream.cuda_stream)
    try:
        lbm.lbm_autotune(lat.ctx, 4)
        info = lat.info()
        lat.step(2 * args.inner)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(MODE_STEPS * args.inner)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        d = lat.diagnostics_all(allow_unstable=True)
    finally:
        lat.close()
    launch_ms = ms / (MODE_STEPS * args.inner)
    algo = BYTES_PER_NODE[storage] * info["fluid_nodes"]
    peak, peak_kind = hbm_peak()
    traffic = committed_traffic(storage, info["nodes"], launch={
        "workload": args.workload, "kernel": step_kernel_name(storage, info), "block_rows": info["block_rows"],
        "grid_blocks": info["grid_blocks"]})
    return {"storage": storage, "value": info["nodes"] * MODE_STEPS * args.inner / (ms / 1e3) / 1e6, "unit": UNIT,
            "launch_ms": launch_ms, "steps_timed": MODE_STEPS * args.inner,
            "roofline": {"bound": "hbm", "achieved": algo / (launch_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": algo / (launch_ms / 1e3) / 1e9 / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "k_step", "algorithmic_bytes_per_launch": algo},
            "launch": {"block_threads": info["block_threads"], "block_rows": info["block_rows"],
                       "grid_blocks": info["grid_blocks"], "wall_inline": info["wall_inline"]},
            "unstable_cases": sum(x["unstable"] for x in d)}


MODE_STEPS = 5


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2505_22256_gb300 import lbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    def barrier():
        if world > 1:
            dist.barrier()

    if args.split:  # the same cases on every rank (rank 0's seeds), each rank stepping its share
        cases, desc = workload(args, 0)
        cases, job_nodes = shard(cases, rank, world)
        weight = 1
    else:
        cases, desc = workload(args, rank)
        job_nodes = None
        weight = world
    surfaces = [c.surface for c in cases]
    stream = torch.cuda.Stream()
    lat = lbm.Lattice(cases, storage=args.storage, cuda_stream=stream.cuda_stream)
    if args.launch_table:
        return launch_table(args, lat, stream)
    # launch shape (row-chunk height, wall-list path) picked by the library's autotuner on the live
    # state, before the timed region
    tuned_ms = None if args.no_autotune else lbm.lbm_autotune(lat.ctx, 4)
    if args.no_autotune and args.wall_inline is not None:
        lbm.lbm_set_wall_path(lat.ctx, args.wall_inline)
    info = lat.info()
    nodes = info["nodes"]
    fluid = info["fluid_nodes"]
    if job_nodes is None:
        job_nodes = nodes  # per rank; weight = world counts every rank's copy

    def contact_angles():  # theta per case; NaN (reported as null) without a surface or an interface
        return lat.contact_angle_all(surfaces)[0]

    def bench_step(ev_pairs=None):
        if ev_pairs is not None:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
        lat.step(args.inner)
        if ev_pairs is not None:
            ev[1].record(stream)
        lat.diagnostics_all(allow_unstable=True)
        if ev_pairs is not None:
            ev[2].record(stream)
        contact_angles()
        if ev_pairs is not None:
            ev[3].record(stream)
            ev_pairs.append(ev)

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    pairs = []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    t0.record(stream)
    for _ in range(args.steps):
        bench_step(pairs)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(t0.elapsed_time(t1), world, "cuda")
    step_ms = sum(e[0].elapsed_time(e[1]) for e in pairs)
    phase_ms = {"time_steps": step_ms / args.steps,
                "diagnostics": sum(e[1].elapsed_time(e[2]) for e in pairs) / args.steps,
                "contact_angle": sum(e[2].elapsed_time(e[3]) for e in pairs) / args.steps}
    ms_per_step = total_ms / args.steps
    value = job_mlups(weight, job_nodes, args.inner * args.steps, total_ms)
    launch_ms = step_ms / (args.inner * args.steps)
    algo_bytes = BYTES_PER_NODE[args.storage] * fluid
    achieved = algo_bytes / (launch_ms / 1e3) / 1e9
    peak, peak_kind = hbm_peak()
    traffic = committed_traffic(args.storage, nodes, launch={
        "workload": args.workload, "kernel": step_kernel_name(args.storage, info), "block_rows": info["block_rows"],
        "grid_blocks": info["grid_blocks"]})
    dall = lat.diagnostics_all(allow_unstable=True)
    d = dall[0]
    theta = [None if th != th else float(th) for th in contact_angles()]

    # e2e through the public API with host buffers: densities in (H2D), 100 steps, fields out (D2H)
    e2e = None
    if not args.no_e2e:
        # all cases back to back in case order, in pinned host memory: one copy per array and
        # direction per bench step through the batched calls
        pin = lambda n: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        total = sum(c.nx * c.ny for c in cases)
        hin = (pin(total), pin(total))
        hin[0][...] = np.concatenate([c.rhoA0.ravel() for c in cases])
        hin[1][...] = np.concatenate([c.rhoB0.ravel() for c in cases])
        hout = [pin(total) for _ in range(4)]
        ksteps = max(2, args.steps)  # as many bench steps as the device-timed region

        # each bench step: densities in, time steps, fields out, enqueued through the overlapped
        # calls, whose copies run on the context's copy streams beside the time steps; the timed
        # region ends when every copy of the last step has landed in host memory
        def e2e_step():
            lbm.lbm_set_densities_all_async(lat.ctx, hin[0], hin[1])
            lat.step(args.inner)
            lbm.lbm_fields_all_async(lat.ctx, *hout)

        def timed(body):
            body()  # first use: staging buffers, streams, graphs
            lat.sync()
            torch.cuda.synchronize()
            barrier()
            t = time.perf_counter()
            for _ in range(ksteps):
                body()
            lat.sync()
            torch.cuda.synchronize()
            barrier()
            return max_over_ranks(time.perf_counter() - t, world, "cuda")

        el = timed(e2e_step)
        h2d = sum(2 * c.nx * c.ny * 8 for c in cases)
        d2h = sum(4 * c.nx * c.ny * 8 for c in cases)

        # the same through the blocking calls (each returns when its copies are done)
        def e2e_blocking():
            lbm.lbm_set_densities_all(lat.ctx, hin[0], hin[1], False)
            lat.step(args.inner)
            lbm.lbm_fields_all(lat.ctx, *hout)

        el_b = timed(e2e_blocking)

        # a continuing run: no re-initialisation, the fields of every case come out after each
        # bench step's time steps (how a long run is monitored)
        def e2e_continuing():
            lat.step(args.inner)
            lbm.lbm_fields_all_async(lat.ctx, *hout)

        el_c = timed(e2e_continuing)
        mk = lambda t: job_mlups(weight, job_nodes, args.inner * ksteps, t * 1e3)
        e2e = {"value": mk(el), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ksteps,
               "step": "lbm_set_densities_all_async (pinned host, all cases), lbm_step(%d), lbm_fields_all_async "
                       "(pinned host, all cases); lbm_synchronize after the last" % args.inner,
               "blocking": {"value": mk(el_b), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                            "steps": ksteps, "step": "lbm_set_densities_all, lbm_step(%d), lbm_fields_all (each host "
                                                     "call waits for its copies)" % args.inner},
               "continuing": {"value": mk(el_c), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
                              "steps": ksteps,
                              "step": "lbm_step(%d), lbm_fields_all_async (pinned host, all cases), no "
                                      "re-initialisation" % args.inner}}

    # step kernels (+ the sliding-wall fix-up after each step where walls slide) + (fields pass +
    # per-case reductions) + batched contact angle (one point pass + one fit launch) when any case has
    # a surface; the contact angle's densities come from the diagnostics pass just before it
    sliding = any(tuple(c.u_wall) != (0.0, 0.0) for c in cases)
    launches = args.inner * (2 if sliding else 1) + 2 + (2 if any(sf is not None for sf in surfaces) else 0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong" if args.split else "weak",
        "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": config_dict(args, cases, desc, world, job_nodes if args.split else None),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind, "kernel": "k_step",
                     "algorithmic_bytes_per_launch": algo_bytes, "launch_ms": launch_ms},
        "launch": {"block_threads": info["block_threads"], "block_rows": info["block_rows"],
                   "grid_blocks": info["grid_blocks"], "work_items": info["work_items"],
                   "wall_inline": info["wall_inline"], "autotuned": tuned_ms is not None,
                   "autotune_best_ms": tuned_ms},
        "e2e": e2e, "gpu_launches": launches * args.steps, "clocks": clk, "phase_ms_per_step": phase_ms,
        "mflups": world * fluid * args.inner * args.steps / (total_ms / 1e3) / 1e6,
        **({"scheme_comparison": [{"case": c.name, "lambda": c.lam, "scheme": c.scheme, "theta_deg": t,
                                   "umax": x["umax"], "rhoA_min": x["rhoA_min"], "rhoA_max": x["rhoA_max"],
                                   "rhoB_min": x["rhoB_min"], "rhoB_max": x["rhoB_max"]}
                                  for c, t, x in zip(cases, theta, dall)]}
           if args.workload == "compare" else {}),
        "sample_diagnostics": {"theta_deg": theta if len(theta) <= 8 else
                               {"measured": sum(t is not None for t in theta),
                                "min": min((t for t in theta if t is not None), default=None),
                                "max": max((t for t in theta if t is not None), default=None)},
                               "case0_umax": d["umax"], "unstable_cases": sum(x["unstable"] for x in dall)},
    }
    lat.close()
    modes = args.storage == "f32" and world == 1 and not args.no_modes
    if modes:  # the FP16 storage form of the same workload (the metric reports it beside FP32)
        line["storage_modes"] = {st: storage_mode_line(args, cases, st, stream) for st in ("f16",)}
    if rank == 0:
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline(args, args.cpu_seconds, parity=True,
                                                also=("f16",) if modes else ())
        elif not args.no_cpu:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------------------
# the 3-D workload (Sec. 3.5): one 200x200x280 lattice per GPU
# ------------------------------------------------------------------------------------------------
def sphere3d_case(args, rank=0):
    from paper_2505_22256_gb300 import scenarios as S

    if args.size:  # the geometry scaled to n x n x 1.4 n
        return S.sphere_droplet_3d_small(int(args.size), lam=1.0, seed=9 + 1000 * rank)
    return S.sphere_droplet_3d(lam=1.0, seed=9 + 1000 * rank)


def cpu_baseline_3d(seconds: float, storage: str | None = None) -> dict:
    """The 3-D FP64 oracle timed on the Sec. 3.5 geometry scaled to 64 x 64 x 90.  storage: also run
    that lattice on the GPU and report its error against the oracle after PARITY_STEPS steps."""
    import numpy as np

    from oracle import d3
    from paper_2505_22256_gb300 import scenarios as S

    sc = S.sphere_droplet_3d_small(64)  # the same geometry scaled to 64 x 64 x 90
    nz, ny, nx = sc.shape
    p = sc.params()
    cfg = d3.Config3(nx, ny, nz, scheme=p["scheme"], tau=p["tau"], G=p["G"], lam=p["lam"], Gw2=p["Gw2"],
                     delta=p["delta"], g=p["g"], second_layer=p["second_layer"],
                     adhesion_stencil=p["adhesion_stencil"])
    f = d3.init3(cfg, sc.solid, sc.rhoA0, sc.rhoB0)
    need = PARITY_STEPS if storage else 1
    snap = None
    n, t0 = 0, time.perf_counter()
    while True:
        f = d3.run3(cfg, sc.solid, f, 1)
        n += 1
        if storage and n == PARITY_STEPS:
            snap = f.copy()
        el = time.perf_counter() - t0
        if (el >= seconds and n >= need) or n >= 10000:
            break
    out = {"value": nx * ny * nz * n / el / 1e6, "unit": UNIT, "cores": cfg.nthreads, "kind": "oracle",
           "sample_s": el, "sample_updates": nx * ny * nz * n,
           "sample": f"the Sec. 3.5 geometry scaled to {nx}x{ny}x{nz}, {n} FP64 time steps in {el:.1f} s on "
                     f"{cfg.nthreads} host threads", "host": host_info()}
    if storage and snap is not None:
        from paper_2505_22256_gb300 import lbm3d

        o = d3.fields3(cfg, sc.solid, snap)
        lat = lbm3d.Lattice3(sc.solid, sc.rhoA0, sc.rhoB0, p, storage)
        lat.step(PARITY_STEPS)
        g = lat.fields()
        lat.close()
        fl = sc.solid == 0
        err_rho = max(float(np.max(np.abs(g[k] - o[k])[fl] / o[k][fl])) for k in (0, 1))
        err_u = max(float(np.max(np.abs(g[k] - o[k])[fl])) for k in (2, 3, 4))
        out["parity"] = parity_record(storage, f"sphere droplet {nx}x{ny}x{nz}", err_rho, err_u)
    return out


def run_ours_3d(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2505_22256_gb300 import lbm3d

    if args.storage not in BYTES_PER_NODE_3D:
        raise SystemExit("the 3-D workload runs in f32, f64, f16 or bf16")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    sc = sphere3d_case(args, rank)
    stream = torch.cuda.Stream()
    lat = lbm3d.Lattice3(sc.solid, sc.rhoA0, sc.rhoB0, sc.params(), args.storage, cuda_stream=stream.cuda_stream)
    nodes = int(sc.solid.size)
    fluid = int((sc.solid == 0).sum())

    def barrier():
        if world > 1:
            dist.barrier()

    def bench_step(pairs=None):
        if pairs is not None:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
        lat.step(args.inner)
        if pairs is not None:
            ev[1].record(stream)
        lat.diagnostics(allow_unstable=True)
        if pairs is not None:
            ev[2].record(stream)
        try:
            th = lat.contact_angle(sc.sphere)[0]
        except Exception:
            th = None
        if pairs is not None:
            ev[3].record(stream)
            pairs.append(ev)
        return th

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    pairs = []
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    t0.record(stream)
    theta = None
    for _ in range(args.steps):
        theta = bench_step(pairs)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(t0.elapsed_time(t1), world, "cuda")
    step_ms = sum(e[0].elapsed_time(e[1]) for e in pairs)
    phase_ms = {"time_steps": step_ms / args.steps,
                "diagnostics": sum(e[1].elapsed_time(e[2]) for e in pairs) / args.steps,
                "contact_angle": sum(e[2].elapsed_time(e[3]) for e in pairs) / args.steps}
    launch_ms = step_ms / (args.inner * args.steps)  # one time step: density pass + march pass
    algo = BYTES_PER_NODE_3D[args.storage] * fluid
    peak, peak_kind = hbm_peak()
    d = lat.diagnostics(allow_unstable=True)
    lat.close()

    e2e = None
    if not args.no_e2e:
        k = max(1, args.steps)  # as many steps as the device-timed region
        # densities in from pinned host memory, steps, fields out to pinned host memory
        pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        hin = (pin(sc.solid.shape), pin(sc.solid.shape))
        hin[0][...] = sc.rhoA0
        hin[1][...] = sc.rhoB0
        hout = [pin(sc.solid.shape) for _ in range(5)]
        l2 = lbm3d.Lattice3(sc.solid, sc.rhoA0, sc.rhoB0, sc.params(), args.storage, cuda_stream=stream.cuda_stream)

        # each bench step enqueued through the overlapped calls; the timed region ends when the last
        # step's fields are in host memory
        def e2e_step():
            l2.set_densities_async(hin[0], hin[1])
            l2.step(args.inner)
            l2.fields_async_into(*hout)

        def e2e_blocking():
            l2.set_densities(hin[0], hin[1])
            l2.step(args.inner)
            l2.fields_into(*hout)

        def timed(body):
            body()
            l2.sync()
            torch.cuda.synchronize()
            barrier()
            t = time.perf_counter()
            for _ in range(k):
                body()
            l2.sync()
            torch.cuda.synchronize()
            barrier()
            return max_over_ranks(time.perf_counter() - t, world, "cuda")

        el = timed(e2e_step)
        el_b = timed(e2e_blocking)
        l2.close()
        mk = lambda t: job_mlups(world, nodes, args.inner * k, t * 1e3)
        e2e = {"value": mk(el), "unit": UNIT, "h2d_bytes_per_step": nodes * 16,
               "d2h_bytes_per_step": nodes * 5 * 8, "steps": k,
               "step": "lbm3d_set_densities_async (pinned host), lbm3d_step(%d), lbm3d_fields_async (pinned "
                       "host); lbm3d_synchronize after the last" % args.inner,
               "blocking": {"value": mk(el_b), "unit": UNIT, "h2d_bytes_per_step": nodes * 16,
                            "d2h_bytes_per_step": nodes * 5 * 8, "steps": k,
                            "step": "lbm3d_set_densities, lbm3d_step(%d), lbm3d_fields (each host call waits "
                                    "for its copies)" % args.inner}}

    line = {
        "metric": METRIC, "value": job_mlups(world, nodes, args.inner * args.steps, total_ms), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": {"workload": f"3-D droplet on a sphere, {'x'.join(map(str, sc.shape[::-1]))} per GPU "
                               f"(the Sec. 3.5 geometry, lambda=1, periodic), "
                               f"{args.inner} time steps + diagnostics + contact angle per step",
                   "storage": args.storage, "nodes_per_gpu": nodes, "fluid_nodes_per_gpu": fluid,
                   "inner_steps": args.inner, "parallelism": f"one lattice per GPU x{world} (no collective)",
                   "l2": "inputs larger than L2 (state %.2f GB per buffer)" % (nodes * BYTES_PER_NODE_3D[args.storage] / 2 / 1e9)},
        "roofline": {"bound": "hbm", "achieved": algo / (launch_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": algo / (launch_ms / 1e3) / 1e9 / peak,
                     "traffic": committed_traffic(args.storage, nodes, "k3_step", KERNEL_SOURCES_3D),
                     "peak_kind": peak_kind,
                     "kernel": "k3_rho + k3_march (one time step)", "algorithmic_bytes_per_launch": algo,
                     "launch_ms": launch_ms},
        "e2e": e2e, "gpu_launches": (2 * args.inner + 3 + 9) * args.steps, "clocks": clk, "phase_ms_per_step": phase_ms,
        "mflups": world * fluid * args.inner * args.steps / (total_ms / 1e3) / 1e6,
        "sample_diagnostics": {"theta_deg": theta, "umax": d["umax"], "unstable": d["unstable"]},
    }
    if rank == 0:
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline_3d(args.cpu_seconds, args.storage)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.split and args.workload == "sphere3d":
        raise SystemExit("--split needs a workload of several cases")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "sphere3d":
        return run_ours_3d(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
