#!/usr/bin/env python
"""Throughput of the Cherenkov bunch hot path: bunches generated and
propagated per second, FP32-bulk and FP64 paths, against the ALU roofline.

Workload (default): 256 showers (primary energies log-uniform 10 GeV -
10 TeV, zenith 0-40 deg), 2e8 e+- steps in one persistent launch replayed
from its captured CUDA graph, 100 telescope spheres over 2 x 2 km, refraction
tables 1000 x 64 up to 70 deg (seeded, synthetic: see workloads/).  A step of
the benchmark is one launch over all 2e8 steps: every bunch generated,
refracted, propagated, tested against the spheres and the crossings
compacted.  The same line carries the 20 TeV shower at 60 deg (1e8 steps,
tables 4000 x 256 to 75 deg) and the 1 TeV vertical shower (2e6 steps) as
legs with their own roofline, and the FP64 path of each.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank simulates its own showers (independent
showers: weak scaling, no collective on the data path); the value is the
bunches of all ranks over the slowest rank's time.  `--impl reference`
times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Cherenkov bunches generated+propagated/s (FP32 vs FP64 path), % of roofline"
WORKLOAD_TEXT = {
    "vertical_1tev": "vertical_1tev: 1 TeV vertical gamma-like shower, 2e6 e+- steps per GPU, "
                     "19 spheres (R 6-12 m, hex 120 m), tables 1000 x 64 to 70 deg, h_obs 2.2 km",
    "inclined_20tev": "inclined_20tev: 20 TeV shower at 60 deg zenith, 1e8 steps per GPU, "
                      "100 spheres over 2 x 2 km, tables 4000 x 256 to 75 deg",
    "batched_256": "batched_256: 256 showers (10 GeV - 10 TeV, zenith 0-40 deg), 2e8 steps per "
                   "GPU in one persistent launch replayed from its CUDA graph, 100 spheres over "
                   "2 x 2 km, tables 1000 x 64 to 70 deg",
}
UNIT = "bunches/s"
WORKLOAD = "batched_256"

# ---------------------------------------------------------------------------
# Algorithmic operation counts, from the algorithm as the oracle states it
# (each add, mul, fma, compare, select, convert, shift or logic op = 1; each
# sqrt, rsqrt or reciprocal = 1; implementation overhead excluded), with the
# work that depends only on the step counted once per step and the work that
# depends only on the launch (the Philox key schedule, 18 adds) not counted.
# Per bunch, FP32/INT32 lane operations of the single-precision path by
# stage; per step, the same for the step's own work.
# ---------------------------------------------------------------------------
OPS_PER_BUNCH_FP32 = {
    "sub_step_loop": 2,
    "philox4x32_10": 71,        # rounds 3-10: 8 x (2 mul.lo + 2 mul.hi + 4 xor); rounds
                                # 1-2: the bunch index's share (M1 j: 2 mul + 1 xor; M0 of
                                # round 1's word 0: 2 mul + 2 xor)
    "deviates": 9,              # 3 x (shift, convert, fma)
    "emission": 36,             # sub-step fraction, sin/cos of the azimuth, cone, lambda, height
    "rare_conditions": 3,
    "n_lookup_snell": 17,       # fine-table lookup, Snell ratio, sin^2, cos
    "tables": 24,               # two indices, two fractions, 2 x bilinear
    "ground_point_time": 21,    # sec, tan, offsets, X, Y, t, direction cosines
    "grid_and_sphere": 24,      # grid cell, one line-sphere test
    "output_counters": 8,       # amortised compaction and counters
}
OPS_PER_BUNCH = sum(OPS_PER_BUNCH_FP32.values())          # 215
OPS_PER_STEP_FP32 = {
    "validity": 11,             # nine finiteness tests, len >= 0, E_kin > 0
    "yield": 50,                # n(h) lookup, sin^2, N / B, its rounding bound, ceil
    "philox_step_share": 8,     # rounds 1-2: the step index's share (2 x (2 mul + 2 xor))
    "step_constants": 32,       # 5 roundings, 2 FP64 differences, azimuth basis, cone,
                                # 1/nb, 1/(beta c), photons per bunch
    "scan": 12,                 # the tile's prefix sum of nb, per step
}
OPS_PER_STEP = sum(OPS_PER_STEP_FP32.values())            # 113
# the floating-point part (everything but Philox), which the FP64 path runs
# on the FP64 pipe, per bunch and per step (the yield chain, 34, and the
# step constants, 30, in FP64)
FP64_OPS_PER_BUNCH = OPS_PER_BUNCH - OPS_PER_BUNCH_FP32["philox4x32_10"]     # 144
FP64_OPS_PER_STEP = 64
FP32_LANES_PER_SM = 128
FP64_FMA_PER_SM_CLK = 2         # GB300: 1/64 of the FP32 rate (ncu: 2 DFMA/cycle/SM)

# DRAM bytes (read + write) per step of one FP32 launch, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum of the fused kernel, in the
# launch shape the autotuner picks for the workload) at 2e6 steps, scaled to a launch
# by its steps (the inputs, 64 B per step, dominate and scale with them).
# Reported only while the kernel sources hash to what was profiled.
TRAFFIC_PER_STEP = {
    "vertical_1tev": (77.26, "e12d0db1d7ddc53f"),      # 128.74 + 25.79 MB at 2e6 steps, 128 x 8
    "inclined_20tev": (74.38, "e12d0db1d7ddc53f"),     # 135.36 + 13.40 MB at 2e6 steps, 128 x 10
    "batched_256": (75.45, "e12d0db1d7ddc53f"),        # 132.56 + 18.35 MB at 2e6 steps, 128 x 10
}
KERNEL_SOURCES = ("cher_kernels.cu", "cher_device.cuh", "cher_internal.h")


def _kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2006_14927_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(workload: str, steps: int):
    t = TRAFFIC_PER_STEP.get(workload)
    if t is None or _kernel_hash() != t[1]:
        return None
    return int(round(t[0] * steps))


def alu_roofline(bunches: float, steps: float, ms: float, sm_count: int, mhz: float):
    """FP32-path roofline: algorithmic lane operations per launch over the
    mean launch time, against the FP32/INT32 lanes x clock (an issue-rate
    bound derived from the unit counts, not a measured peak)."""
    ops = OPS_PER_BUNCH * bunches + OPS_PER_STEP * steps
    peak = sm_count * FP32_LANES_PER_SM * mhz * 1e6
    achieved = ops / (ms / 1e3)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
            "frac": achieved / peak, "ops_per_bunch": OPS_PER_BUNCH,
            "ops_per_step": OPS_PER_STEP, "launch_ms": ms,
            "peak_source": f"derived: {sm_count} SMs x {FP32_LANES_PER_SM} FP32/INT32 lanes x "
                           f"{mhz:.0f} MHz max clock (issue-rate bound)"}


def fp64_roofline(bunches: float, steps: float, ms: float, sm_count: int, mhz: float):
    """FP64-path roofline: the floating-point operations on the FP64 pipe."""
    ops = FP64_OPS_PER_BUNCH * bunches + FP64_OPS_PER_STEP * steps
    peak = sm_count * FP64_FMA_PER_SM_CLK * mhz * 1e6
    achieved = ops / (ms / 1e3)
    return {"bound": "fp64", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
            "frac": achieved / peak, "ops_per_bunch": FP64_OPS_PER_BUNCH,
            "ops_per_step": FP64_OPS_PER_STEP,
            "peak_source": f"derived: {sm_count} SMs x {FP64_FMA_PER_SM_CLK} FP64 lanes x "
                           f"{mhz:.0f} MHz"}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the
    timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t_load=None):
        rows = []
        try:
            for ln in open(self.path):
                f = [x.strip() for x in ln.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def shard(rank: int, n_per_rank: int, base_seed: int):
    """Weak scaling: rank r simulates its own shower (seed base + r) and
    numbers its steps from r * n_per_rank, so no two ranks share a Philox
    counter and no collective is needed on the data path."""
    return base_seed + rank, rank * n_per_rank


def reduce_over_ranks(t_local: float, bunches_local: float, world: int, device):
    """Whole-job figures: the slowest rank's time and the bunches of all
    ranks (the only collectives of the benchmark, outside the timed work)."""
    if world <= 1:
        return t_local, bunches_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    b = torch.tensor([bunches_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), float(b.item())


def _sample_workload(workload: str, n: int = 20_000):
    """A bounded sample of a workload for the CPU oracle: its generator at n
    steps (the 256-shower batch keeps its 256 showers, with n steps split
    among them in proportion to energy as in the full batch)."""
    import workloads
    if workload == "batched_256":
        return workloads.batched_256(total=n), f"the 256 showers of batched_256 with {n} steps"
    if workload in ("plain_fp64", "adjoint_300gev"):
        sc = workloads.WORKLOADS[workload]()
        return sc, f"{workload}: all {len(sc['tracks']['x0'])} steps"
    return workloads.WORKLOADS[workload](n=n), f"{workload}: its first {n} steps"


def run_reference(args):
    """The FP64 CPU oracle on a bounded sample of the same workload."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import oracle
    oracle.build()
    sc, what = _sample_workload(args.workload)
    M = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"], H=sc["H"],
                     Z=sc["Z"], theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"])
    tr = sc["tracks"]
    for _ in range(args.warmup):
        M.bunches(tr, 7)
    t0 = time.perf_counter()
    nb = 0
    for _ in range(args.steps):
        o = M.bunches(tr, 7)
        nb += len(o["status"])
    dt = time.perf_counter() - t0
    v = nb / dt
    cores = oracle.num_threads()
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{args.workload} sample: {what}",
                       "precision": "fp64 oracle (table variant)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{what} ({nb // args.steps} bunches) per step, "
                                       f"OpenMP over steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _make_workload(wl: str, scale: float, rank: int):
    import workloads
    if wl == "vertical_1tev":
        n_req = int(2_000_000 * scale)
        seed, track_base = shard(rank, n_req, 2)
        return workloads.vertical_1tev(n=n_req, seed=seed), track_base
    if wl == "inclined_20tev":
        n_req = int(100_000_000 * scale)
        seed, track_base = shard(rank, n_req, 5)
        return workloads.inclined_20tev(n=n_req, seed=seed), track_base
    if wl == "batched_256":
        n_req = int(200_000_000 * scale)
        seed, track_base = shard(rank, n_req, 3)
        return workloads.batched_256(total=n_req, seed=seed), track_base
    sc = workloads.WORKLOADS[wl]()
    return sc, rank * len(sc["tracks"]["x0"])


def _cap(wl: str, scale: float, cap_arg):
    """Records per telescope: the densest telescope of each workload fits
    (the batch: 12e6 x 100 telescopes x 40 B = 48 GB of the 288 GB)."""
    if cap_arg:
        return cap_arg
    full = {"vertical_1tev": 600_000, "batched_256": 12_000_000}.get(wl, 8_000_000)
    return full if wl == "vertical_1tev" else max(200_000, int(full * scale))


class Bench:
    """Timing of one workload on one context (CUDA events on the launching
    stream, L2 flushed by a 256 MiB write between timed launches)."""

    def __init__(self, P, dev, sc, wl, scale, cap, track_base, barrier):
        import torch
        self.P, self.dev, self.sc, self.wl = P, dev, sc, wl
        self.track_base, self.barrier, self.cap = track_base, barrier, cap
        self.n = len(sc["tracks"]["x0"])
        t0 = time.perf_counter()
        self.ctx = P.Context(sc["atm"], sc["h_obs"], sc["telescopes"])
        self.ctx.build_refraction_tables(sc["H"], sc["Z"], sc["theta_max_deg"], sc["h_max"])
        self.table_s = time.perf_counter() - t0
        self.flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.current_stream()
        self.bufs = {}

    def buffers(self, prec):
        if prec not in self.bufs:
            P = self.P
            dtr = P.device_tracks(self.sc["tracks"], prec, device=self.dev, t_ref=self.sc["t_ref"])
            self.bufs[prec] = (dtr, self.ctx.alloc_hits(self.cap, prec, device=self.dev))
        return self.bufs[prec]

    def release(self, prec):
        import torch
        self.bufs.pop(prec, None)
        torch.cuda.empty_cache()

    def measure(self, prec, steps, warmup, launch=None, graph=False, prof=None):
        """Mean-free list of per-launch times (ms), the stats of the last
        launch and the wall time of the timed loop."""
        import torch
        dtr, out = self.buffers(prec)
        ctx = self.ctx
        pkw = {} if prof is None else dict(profile=prof[0], bin_gcm2=prof[1], axis_cos=prof[2])
        if launch is not None:
            ctx.set_launch(*launch)

        def once():
            ctx.generate_propagate(dtr, 11, prec, out, track_base=self.track_base, **pkw)

        g = None
        if graph:
            g = ctx.graph(dtr, 11, prec, out, track_base=self.track_base)
            once = g.launch                      # noqa: F811 (the graph replaces the call)
        for _ in range(warmup):
            once()
        code, stats = ctx.sync_status(out)
        if code not in (0, 6):                   # 6: a buffer overflowed (counted)
            raise RuntimeError(f"status {code} in warm-up")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        self.barrier()
        w0 = time.perf_counter()
        for k in range(steps):
            self.flush.fill_(k & 0xff)           # evict L2 between timed launches
            ev[k][0].record(self.stream)
            once()
            ev[k][1].record(self.stream)
        self.barrier()
        wall = time.perf_counter() - w0
        ms = [a.elapsed_time(b) for a, b in ev]
        code, stats = ctx.sync_status(out)
        if g is not None:
            g.close()
        return dict(ms=ms, wall=wall, stats=stats, code=code)


def workload_leg(P, dev, wl, scale, cap_arg, steps, warmup, launch, main_launch, sm_count, mhz,
                 barrier):
    """One more workload in the same run: FP32 (its own autotuned launch
    shape, or the one given; regular launches) and FP64 (the main workload's
    shape), each with its roofline."""
    import torch
    sc, tb = _make_workload(wl, scale, 0)
    B = Bench(P, dev, sc, wl, scale, _cap(wl, scale, cap_arg), tb, barrier)
    if launch is None:
        dtr, out = B.buffers(P.CHER_FP32_BULK)
        B.ctx.autotune(dtr, 11, P.CHER_FP32_BULK, out)
    own = launch if launch is not None else B.ctx.get_launch()
    r32 = B.measure(P.CHER_FP32_BULK, steps, warmup, launch=own)
    B.release(P.CHER_FP32_BULK)
    r64 = B.measure(P.CHER_FP64, max(3, steps // 4), 3, launch=main_launch)
    B.release(P.CHER_FP64)
    n = B.n
    b32, b64 = float(r32["stats"][3]), float(r64["stats"][3])
    ms32, ms64 = statistics.mean(r32["ms"]), statistics.mean(r64["ms"])
    rl = alu_roofline(b32, n, ms32, sm_count, mhz)
    rl["traffic"] = _traffic(wl, n)
    res = {"value": b32 / (ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32,
           "bunches_per_step": int(b32), "steps_per_gpu": n, "roofline": rl,
           "fp64": {"value": b64 / (ms64 / 1e3), "ms_per_step": ms64,
                    "roofline": fp64_roofline(b64, n, ms64, sm_count, mhz)},
           "fp32_over_fp64": (b32 / ms32) / (b64 / ms64),
           "overflowed_records": int(r32["stats"][10]), "table_build_s": B.table_s,
           "launch": {"block": own[0], "ctas_per_sm": own[1]},
           "workload": WORKLOAD_TEXT.get(wl, wl)}
    B.ctx.close()
    del B
    torch.cuda.empty_cache()
    return res


def _leg(fn, *a):
    """A secondary leg of the line: its result, or the error it raised (the
    headline and the other legs are still reported)."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 - reported in the line, not swallowed
        print(f"leg {fn.__name__} failed: {e!r}", file=sys.stderr, flush=True)
        return {"error": f"{type(e).__name__}: {e}"[:300]}


def run_ours(args):
    import torch

    import paper_2006_14927_gb300 as P
    import workloads

    rank, world, local = _env_rank()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    P.build()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- workload (each rank its own showers: weak scaling) ---------------
    wl = args.workload
    sc, track_base = _make_workload(wl, args.scale, rank)
    cap = _cap(wl, args.scale, args.cap)
    B = Bench(P, dev, sc, wl, args.scale, cap, track_base, barrier)
    ctx, n = B.ctx, B.n
    steps, warmup = args.steps, args.warmup
    FP32, FP64 = P.CHER_FP32_BULK, P.CHER_FP64

    # autotuned launch shape (or the one given), then the headline: the
    # persistent launch replayed from its captured graph
    qprec = FP64 if (args.quick and args.prec == "fp64") else FP32
    dtr_q, out_q = B.buffers(qprec)
    if args.launch is not None:
        ctx.set_launch(*(int(v) for v in args.launch.split(",")))
    else:
        ctx.autotune(dtr_q, 11, qprec, out_q)
    launch = ctx.get_launch()
    table_s = B.table_s
    gpu = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
    with ClockSampler(int(gpu) if gpu.isdigit() else 0) as clk:
        rg = B.measure(qprec, steps, warmup, graph=not args.quick)
    clocks = clk.summary()
    if args.sweep and rank == 0:
        for shape in [(128, 1), (128, 2), (128, 4), (128, 6), (128, 8), (256, 1), (256, 2),
                      (256, 3), (256, 4), (512, 1), (512, 2), (128, 0), (256, 0)]:
            r = B.measure(FP32, 5, 2, launch=shape)
            t = statistics.median(r["ms"])
            print(json.dumps({"sweep": shape, "ms": t,
                              "bunches_per_s": float(r["stats"][3]) / (t / 1e3)}), flush=True)
        ctx.set_launch(*launch)
    if args.quick:
        t = sum(rg["ms"]) / 1e3
        if rank == 0:
            print(json.dumps({"quick": True, "workload": wl,
                              "value": float(rg["stats"][3]) * len(rg["ms"]) / t,
                              "unit": UNIT, "ms_per_step": 1e3 * t / len(rg["ms"]),
                              "launch": launch, "clocks": clocks}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    # the same launch without the graph (one C-ABI call per launch)
    r32 = B.measure(FP32, steps, 3, launch=launch)
    # the longitudinal production profile (CERLDE) in the same launch:
    # 10 g/cm^2 bins to 2000 g/cm^2 of slant depth, one row per shower
    legs_steps = max(3, steps // 4)
    n_rows = max(len(sc["t_ref"]), 1)
    prof_t = torch.zeros((n_rows, 200), dtype=torch.float64, device=dev)
    axis_cos = np.cos(np.asarray(sc.get("axis_zenith_rad", np.zeros(n_rows)), float))
    r32p = B.measure(FP32, legs_steps, 3, prof=(prof_t, 10.0, axis_cos))
    # the atmospheric transmission draw (synthetic Rayleigh + aerosol table)
    ctx.set_transmission(workloads.synthetic_transmission(h_obs=sc["h_obs"], h_max=sc["h_max"]))
    r32t = B.measure(FP32, legs_steps, 3)
    ctx.set_transmission(None)
    # the wavelength-dependent index (Edlen's dispersion of standard air, 9 nodes)
    ctx.set_dispersion(workloads.synthetic_dispersion(lambda1_nm=sc["lambda1_nm"],
                                                      lambda2_nm=sc["lambda2_nm"]))
    r32d = B.measure(FP32, legs_steps, 3)
    ctx.set_dispersion(None)
    ctx.set_launch(*launch)
    # the FP64 path (its own buffers; the batch's FP64 records take 96 GB)
    r64 = B.measure(FP64, legs_steps, 3)
    B.release(FP64)

    def total(r):
        return reduce_over_ranks(sum(r["ms"]) / 1e3, float(r["stats"][3]) * len(r["ms"]),
                                 world, dev)

    tg, bg = total(rg)
    t32, b32 = total(r32)
    t64, b64 = total(r64)
    vg, v32, v64 = bg / tg, b32 / t32, b64 / t64

    # ---- end to end: host buffers through the C ABI ---------------------
    # (one process: a failure is reported in the line; several: every rank
    # must reach the same barriers, so an error ends the run)
    e2e = None if args.no_e2e else (
        _leg(e2e_leg, P, B, r32, steps, warmup, world, dev) if world == 1
        else e2e_leg(P, B, r32, steps, warmup, world, dev))
    B.release(FP32)

    peaks, src = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    legs = {}
    if world == 1 and not args.no_legs and wl == "batched_256" and args.scale == 1.0:
        ctx.close()
        del B, ctx
        torch.cuda.empty_cache()
        for other in ("inclined_20tev", "vertical_1tev"):
            given = tuple(int(v) for v in args.launch.split(",")) if args.launch else None
            legs[other] = _leg(workload_leg, P, dev, other, 1.0, None, steps, warmup, given,
                               launch, sm_count, mhz, barrier)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (ALU bound) ----------------------
    st = rg["stats"]
    bunches, steps_n = float(st[3]), float(st[0])
    ms_g = statistics.mean(rg["ms"])
    rl = alu_roofline(bunches, steps_n, ms_g, sm_count, mhz)
    rl["traffic"] = _traffic(wl, n) if args.scale == 1.0 else None
    ms64 = statistics.mean(r64["ms"])
    rl64 = fp64_roofline(float(r64["stats"][3]), steps_n, ms64, sm_count, mhz)
    # the FP64 path beside the FP32 one inside the roofline object as well
    rl["fp64_path"] = {"value": v64, "frac": rl64["frac"], "fp32_over_fp64": vg / v64}
    cpu = _leg(cpu_baseline, wl) if world == 1 else None
    line = {
        "metric": METRIC, "value": vg, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": 1e3 * tg / len(rg["ms"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "fp64": {"value": v64, "unit": UNIT, "ms_per_step": 1e3 * t64 / len(r64["ms"]),
                 "steps": len(r64["ms"]), "roofline": rl64},
        "fp32_over_fp64": vg / v64,
        "gpu_launches": len(rg["ms"]),
        "config": {"workload": WORKLOAD_TEXT.get(wl, wl) +
                               (f" (scale {args.scale})" if args.scale != 1.0 else ""),
                   "steps_per_gpu": n, "n_showers": int(len(sc["t_ref"])),
                   "precision": "fp32_bulk (FP64 yield)", "bunches_per_step": int(bunches),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "launch": {"block": launch[0], "ctas_per_sm": launch[1],
                              "persistent": launch[1] > 0, "graph": True},
                   "table_build_s": table_s},
        "roofline": rl,
        "clocks": clocks,
        "e2e": e2e,
        "regular_launch": {"value": v32, "ms_per_step": 1e3 * t32 / len(r32["ms"]),
                           "note": "one cher_generate_propagate call per launch, no graph"},
        "overflowed_records": int(rg["stats"][10]),
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    ms32 = statistics.mean(r32["ms"])
    line["features"] = {
        "profile": {"overhead": statistics.mean(r32p["ms"]) / ms32 - 1.0,
                    "bins": int(prof_t.shape[1]), "bin_gcm2": 10.0, "rows": n_rows},
        "transmission": {"overhead": statistics.mean(r32t["ms"]) / ms32 - 1,
                         "absorbed_frac": float(r32t["stats"][11]) / float(r32t["stats"][3])},
        "dispersion": {"overhead": statistics.mean(r32d["ms"]) / ms32 - 1,
                       "value": float(r32d["stats"][3]) / (statistics.mean(r32d["ms"]) / 1e3)}}
    for k, v in legs.items():
        line[k] = v
    if world == 1 and not args.no_legs and wl == "batched_256" and args.scale == 1.0:
        line["adjoint"] = _leg(adjoint_leg, dev, steps)
        if "error" not in line["adjoint"]:
            line["adjoint"]["cpu_baseline"] = _leg(cpu_baseline_readout)
        line["e2e_generated"] = _leg(generated_leg, P, dev, steps, warmup)
    # the headline figures once more at the end of the line
    line["summary"] = {"fp32": vg, "fp32_frac": rl["frac"], "fp64": v64,
                       "fp64_frac": rl64["frac"], "fp32_over_fp64": vg / v64,
                       **{f"{k}_fp32_frac": v["roofline"]["frac"] for k, v in legs.items()
                          if "error" not in v},
                       **{f"{k}_fp64_frac": v["fp64"]["roofline"]["frac"] for k, v in legs.items()
                          if "error" not in v}}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_leg(args):
    """One secondary leg alone: the step generator (2e6 steps of the 1 TeV
    vertical shower), the adjoint (300 GeV shower, both precisions), the
    beyond-table fallback or the end to end from shower parameters."""
    import torch

    import paper_2006_14927_gb300 as P
    import workloads
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if args.leg == "adjoint":
        print(json.dumps({"leg": "adjoint", **adjoint_leg(dev, args.steps)}), flush=True)
        return
    if args.leg == "fallback":
        print(json.dumps({"leg": "fallback", **fallback_leg(dev, args)}), flush=True)
        return
    if args.leg == "e2e_generated":
        print(json.dumps({"leg": "e2e_generated",
                          **generated_leg(P, dev, args.steps, args.warmup)}), flush=True)
        return
    sc = workloads.vertical_1tev(n=10)
    ctx = P.Context(sc["atm"], sc["h_obs"], sc["telescopes"])
    showers = [dict(e0_mev=1.0e6, zenith=0.0, azimuth=0.0, core_x=0.0, core_y=0.0, n=2_000_000)]
    for _ in range(args.warmup):
        ctx.generate_steps(showers, 11, P.CHER_FP32_BULK)
    ms = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.generate_steps(showers, 11, P.CHER_FP32_BULK)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    print(json.dumps({"leg": "generator", "ms_per_call": t, "steps": showers[0]["n"],
                      "GBps_written": showers[0]["n"] * 64 / (t / 1e3) / 1e9}), flush=True)
    ctx.close()


def fallback_leg(dev, args):
    """Large zeniths on the 60-degree shower (2e6 steps, FP32): refraction
    tables to 61 deg with the beyond-table fallback up to 80 deg (about 9 % of
    the bunches arrive past the tables and take the ray integrals), against
    tables to 75 deg that cover every bunch, and the curved atmosphere
    (Earth radius 6371 km) with its tables to 80 deg."""
    import torch

    import paper_2006_14927_gb300 as P
    import workloads
    sc = workloads.inclined_20tev(n=2_000_000)
    dtr = P.device_tracks(sc["tracks"], P.CHER_FP32_BULK, device=dev, t_ref=sc["t_ref"])
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    res = {}
    for name, theta, fb, radius in (("tables_75deg", 75.0, 0.0, 0.0),
                                    ("tables_61deg_fallback_80deg", 61.0, 80.0, 0.0),
                                    ("curved_tables_80deg", 80.0, 0.0, 6.371e6)):
        ctx = P.Context(sc["atm"], sc["h_obs"], sc["telescopes"])
        ctx.set_curved(radius)
        ctx.build_refraction_tables(1000, 64, theta, sc["h_max"])
        ctx.set_fallback(fb)
        out = ctx.alloc_hits(2_000_000, P.CHER_FP32_BULK, device=dev)
        for _ in range(args.warmup):
            ctx.generate_propagate(dtr, 11, P.CHER_FP32_BULK, out)
        ms = []
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.generate_propagate(dtr, 11, P.CHER_FP32_BULK, out)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        code, st = ctx.sync_status(out)
        res[name] = {"ms_per_step": statistics.median(ms), "bunches": int(st[3]),
                     "fallback_bunches": int(st[12]), "angle_drops": int(st[7]),
                     "hits": int(st[9])}
        ctx.close()
    return res


def e2e_leg(P, B, r32, steps, warmup, world, dev):
    """The same metric end to end through the C ABI: every step copies its
    whole input up from pinned host memory and its records, counts and
    statistics back, inside the timed region.  A three-stage pipeline over
    steps: step k+1's inputs go up (copy stream) and step k-1's records come
    down (second copy stream) while step k's kernel runs; two input sets, two
    output buffers and two host record buffers.  Step k-1's download waits
    until step k's kernel has started (a download already in flight when the
    kernel's inputs landed held the kernel back until it ended)."""
    import torch
    sc, ctx, cap, track_base = B.sc, B.ctx, B.cap, B.track_base
    prec = P.CHER_FP32_BULK
    dtr, out = B.buffers(prec)
    host = {k: torch.as_tensor(np.ascontiguousarray(v)).pin_memory()
            for k, v in sc["tracks"].items() if k != "shower"}
    host["ux"], host["uy"], host["uz"] = (host[k].to(torch.float32).pin_memory()
                                          for k in ("ux", "uy", "uz"))
    host["shower"] = torch.as_tensor(
        np.ascontiguousarray(sc["tracks"]["shower"]).view(np.int32)).pin_memory()
    dtr = {k: v for k, v in dtr.items()}
    n_tel = ctx.n_tel
    # host records packed telescope after telescope: room for the crossings
    # of the timed launches (the same seed gives the same records every step;
    # the copies below refuse to truncate)
    n_rec = int(int(r32["stats"][9]) * 1.1) + 4096
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    sets = [dtr, {k: torch.empty_like(v) for k, v in dtr.items()}]
    sets[1]["t_ref"].copy_(dtr["t_ref"])
    outs = [out, ctx.alloc_hits(cap, prec, device=dev)]
    hrec = [tuple(torch.empty(shape, dtype=dt).pin_memory()
                  for shape, dt in (((n_rec, 4), torch.float32), ((n_rec, 4), torch.float32),
                                    (n_rec, torch.int64)))
            for _ in range(2)]
    h_cnts = [torch.empty(n_tel, dtype=torch.int64).pin_memory() for _ in range(2)]
    h_sts = [torch.empty(P.NSTATS, dtype=torch.int64).pin_memory() for _ in range(2)]
    # the records of a step are packed on the device (cher_pack_records)
    # and come down in one copy per array
    pk = [dict(pos=torch.empty((n_rec, 4), dtype=torch.float32, device=dev),
               tim=torch.empty((n_rec, 4), dtype=torch.float32, device=dev),
               key=torch.empty(n_rec, dtype=torch.int64, device=dev),
               offset=torch.empty(n_tel + 1, dtype=torch.int64, device=dev))
          for _ in range(2)]
    h_offs = [torch.empty(n_tel + 1, dtype=torch.int64).pin_memory() for _ in range(2)]
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    comp = torch.cuda.current_stream()
    ev = {k: [torch.cuda.Event(), torch.cuda.Event()]
          for k in ("up", "kern", "cnt", "down", "start")}

    def upload(b):
        with torch.cuda.stream(up):
            up.wait_event(ev["kern"][b])            # the last kernel on set b is done
            for k, v in host.items():
                sets[b][k].copy_(v, non_blocking=True)
            ev["up"][b].record(up)

    def launch_step(b):
        comp.wait_event(ev["up"][b])
        comp.wait_event(ev["down"][b])             # out b's records are down
        ev["start"][b].record(comp)
        ctx.generate_propagate(sets[b], 11, prec, outs[b], track_base=track_base)
        ev["kern"][b].record(comp)
        ctx.pack_records(outs[b], pk[b], stream=comp)
        h_cnts[b].copy_(outs[b].count, non_blocking=True)
        h_sts[b].copy_(outs[b].stats, non_blocking=True)
        h_offs[b].copy_(pk[b]["offset"], non_blocking=True)
        ev["cnt"][b].record(comp)

    def download(b):
        ev["cnt"][b].synchronize()                  # this step's counts on the host
        nbytes = (h_cnts[b].numel() + h_sts[b].numel() + h_offs[b].numel()) * 8
        total = int(h_offs[b][-1])
        if total > n_rec:
            raise RuntimeError("host record buffer too small")
        with torch.cuda.stream(down):
            down.wait_event(ev["cnt"][b])           # the packed records are written
            down.wait_event(ev["start"][1 - b])     # the next step's kernel has started
            hp, ht, hk = hrec[b]
            if total > 0:
                hp[:total].copy_(pk[b]["pos"][:total], non_blocking=True)
                ht[:total].copy_(pk[b]["tim"][:total], non_blocking=True)
                hk[:total].copy_(pk[b]["key"][:total], non_blocking=True)
            nbytes += total * 40
            ev["down"][b].record(down)
        return nbytes

    def run(n_steps):
        nbytes = 0
        upload(0)
        for k in range(n_steps):
            b = k % 2
            if k + 1 < n_steps:
                upload(1 - b)
            launch_step(b)
            if k >= 1:
                nbytes = download(1 - b)
        nbytes = download((n_steps - 1) % 2)
        down.synchronize()
        comp.synchronize()
        return nbytes

    run(max(2, warmup // 2))
    B.barrier()
    e0 = time.perf_counter()
    d2h = run(steps)
    B.barrier()
    te = time.perf_counter() - e0
    te, _ = reduce_over_ranks(te, 0.0, world, dev)
    bunches = float(r32["stats"][3])
    del outs, sets, pk
    return {"value": bunches * steps / te, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "pipelined": "step k+1 up and step k-1 down during step k's kernel "
                         "(each download starts once the next kernel has)"}


def generated_leg(P, dev, steps, warmup):
    """End to end from shower parameters: the 1 TeV vertical shower's 2e6
    steps come from the device generator (cher_generate_steps), only the
    shower parameters and its depth table go up, the packed records come
    down; and the generator alone (64 B of steps written per step).  Two
    stages over steps: step k's generator, kernel and packing run on the
    compute stream while step k-1's records come down on a copy stream (each
    download starts once the next step's work has); two step buffers, two
    output buffers and two host record buffers."""
    import torch

    import workloads
    sc = workloads.vertical_1tev(n=10)
    ctx = P.Context(sc["atm"], sc["h_obs"], sc["telescopes"])
    ctx.build_refraction_tables(sc["H"], sc["Z"], sc["theta_max_deg"], sc["h_max"])
    prec = P.CHER_FP32_BULK
    n = 2_000_000
    showers = [dict(e0_mev=1.0e6, zenith=0.0, azimuth=0.0, core_x=0.0, core_y=0.0, n=n)]
    n_tel = ctx.n_tel
    outs = [ctx.alloc_hits(600_000, prec, device=dev) for _ in range(2)]
    gens = [ctx.generate_steps(showers, 11, prec) for _ in range(2)]
    n_rec = n_tel * 600_000
    pk = [dict(pos=torch.empty((n_rec, 4), dtype=torch.float32, device=dev),
               tim=torch.empty((n_rec, 4), dtype=torch.float32, device=dev),
               key=torch.empty(n_rec, dtype=torch.int64, device=dev),
               offset=torch.empty(n_tel + 1, dtype=torch.int64, device=dev))
          for _ in range(2)]
    hrec = [tuple(torch.empty(shape, dtype=dt).pin_memory()
                  for shape, dt in (((n_rec, 4), torch.float32), ((n_rec, 4), torch.float32),
                                    (n_rec, torch.int64)))
            for _ in range(2)]
    h_cnts = [torch.empty(n_tel, dtype=torch.int64).pin_memory() for _ in range(2)]
    h_sts = [torch.empty(P.NSTATS, dtype=torch.int64).pin_memory() for _ in range(2)]
    h_offs = [torch.empty(n_tel + 1, dtype=torch.int64).pin_memory() for _ in range(2)]
    down = torch.cuda.Stream(device=dev)
    comp = torch.cuda.current_stream()
    ev = {k: [torch.cuda.Event(), torch.cuda.Event()] for k in ("cnt", "down", "start")}

    def launch_step(b):
        comp.wait_event(ev["down"][b])             # out b's records are down
        ev["start"][b].record(comp)
        dg = ctx.generate_steps(showers, 11, prec, out=gens[b])
        ctx.generate_propagate(dg, 11, prec, outs[b])
        ctx.pack_records(outs[b], pk[b], stream=comp)
        h_cnts[b].copy_(outs[b].count, non_blocking=True)
        h_sts[b].copy_(outs[b].stats, non_blocking=True)
        h_offs[b].copy_(pk[b]["offset"], non_blocking=True)
        ev["cnt"][b].record(comp)

    def download(b):
        ev["cnt"][b].synchronize()                  # this step's counts on the host
        nbytes = (h_cnts[b].numel() + h_sts[b].numel() + h_offs[b].numel()) * 8
        total = int(h_offs[b][-1])
        if total > n_rec:
            raise RuntimeError("host record buffer too small")
        with torch.cuda.stream(down):
            down.wait_event(ev["cnt"][b])           # the packed records are written
            down.wait_event(ev["start"][1 - b])     # the next step's work has started
            hp, ht, hk = hrec[b]
            if total > 0:
                hp[:total].copy_(pk[b]["pos"][:total], non_blocking=True)
                ht[:total].copy_(pk[b]["tim"][:total], non_blocking=True)
                hk[:total].copy_(pk[b]["key"][:total], non_blocking=True)
            nbytes += total * 40
            ev["down"][b].record(down)
        return nbytes, int(h_sts[b][3])

    def run(n_steps):
        nbytes, nb = 0, 0
        for k in range(n_steps):
            b = k % 2
            launch_step(b)
            if k >= 1:
                nbytes, got = download(1 - b)
                nb += got
        nbytes, got = download((n_steps - 1) % 2)
        nb += got
        down.synchronize()
        comp.synchronize()
        return nbytes, nb

    run(max(2, warmup // 2))
    g0 = time.perf_counter()
    gd2h, gb = run(steps)
    tg = time.perf_counter() - g0
    gen_buf = gens[0]
    gms = []
    for _ in range(steps):
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record()
        ctx.generate_steps(showers, 11, prec, out=gen_buf)
        b_.record()
        torch.cuda.synchronize()
        gms.append(a_.elapsed_time(b_))
    g_ms = statistics.median(gms)
    peaks_, _src = _peaks()
    g_gbs = n * 64 / (g_ms / 1e3) / 1e9
    ctx.close()
    return {"value": gb / tg, "unit": UNIT, "h2d_bytes_per_step": 64 + 16 + 4 * 1024 + 8,
            "d2h_bytes_per_step": int(gd2h), "steps_generated": n,
            "bunches_per_step": gb // steps,
            "pipelined": "step k-1's records down during step k's generator and kernel",
            "generator": {"ms_per_call": g_ms, "steps_per_s": n / (g_ms / 1e3),
                          "roofline": {"bound": "hbm", "achieved": g_gbs,
                                       "peak": float(peaks_.get("hbm_gbs", 6800.0)),
                                       "unit": "GB/s",
                                       "frac": g_gbs / float(peaks_.get("hbm_gbs", 6800.0)),
                                       "bytes_per_step": 64}}}


def adjoint_leg(dev, steps):
    """The adjoint of the telescope read-out on the 300 GeV shower (1e5
    steps, 19 telescopes, sigma 1 m): screening launch, listed bunch pairs
    recomputed in dual numbers, FP64 gradient atomics.  Unit: bunches of the
    input handled per second of the whole call."""
    import torch

    import paper_2006_14927_gb300 as P
    import workloads
    sc = workloads.adjoint_300gev()
    ctx = P.Context(sc["atm"], sc["h_obs"], sc["telescopes"])
    ctx.build_refraction_tables(sc["H"], sc["Z"], sc["theta_max_deg"], sc["h_max"])
    rng = np.random.default_rng(99)
    n_tel = len(sc["telescopes"])
    gD, gT = rng.normal(0.0, 1.0, n_tel), rng.normal(0.0, 0.05, n_tel)
    res = {}
    for name, prec in (("fp32", P.CHER_FP32_BULK), ("fp64", P.CHER_FP64)):
        dtr = P.device_tracks(sc["tracks"], prec, device=dev, t_ref=sc["t_ref"])
        nb, _ = ctx.segment_yield(dtr, prec)
        bunches = float(nb.to(torch.float64).sum())
        for _ in range(3):
            ctx.adjoint(dtr, 4, prec, gD, gT, 1.0, nb)
        torch.cuda.synchronize()
        ms = []
        for _ in range(max(3, steps // 2)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.adjoint(dtr, 4, prec, gD, gT, 1.0, nb)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        t = statistics.mean(ms)
        res[name] = {"ms_per_call": t, "value": bunches / (t / 1e3), "unit": UNIT}
    res["bunches"] = int(bunches)
    res["steps"] = int(len(sc["tracks"]["x0"]))
    ctx.close()
    return res


def cpu_baseline_readout(n: int = 20000):
    """Beside the adjoint: the oracle's read-out S_k, U_k (the function
    whose gradient the adjoint computes) as it stands, on the first n steps
    of the 300 GeV shower."""
    import oracle
    import workloads
    oracle.build()
    sc = workloads.adjoint_300gev()
    sub = {k: v[:n] for k, v in sc["tracks"].items()}
    M = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"], H=sc["H"],
                     Z=sc["Z"], theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"])
    nb_o, _, _, _ = M.segment_yield(sub)
    t0 = time.perf_counter()
    M.density_sums(sub, 4, nb_o, 1.0)
    dt = time.perf_counter() - t0
    return {"value": float(nb_o.sum()) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"read-out S, U of the first {n} steps ({int(nb_o.sum())} bunches), "
                      f"single-threaded"}


def cpu_baseline(workload: str = WORKLOAD):
    """The oracle as it stands on this host's cores, on a bounded sample of
    the workload (its generator at 20 000 steps), repeated for about 10 s;
    and single-threaded on a fifth of the sample for about 3 s."""
    import oracle
    oracle.build()
    sc, what = _sample_workload(workload)
    M = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], h_max=sc["h_max"], H=sc["H"],
                     Z=sc["Z"], theta_max_deg=sc["theta_max_deg"], t_ref=sc["t_ref"])
    M.bunches(sc["tracks"], 7)
    t0 = time.perf_counter()
    reps, nb = 0, 0
    while time.perf_counter() - t0 < 10.0 or reps < 2:
        o = M.bunches(sc["tracks"], 7)
        nb += len(o["status"])
        reps += 1
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    res = {"value": nb / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{what} ({nb // reps} bunches), repeated {reps} times, "
                     f"FP64 table variant, OpenMP over steps"}
    n = len(sc["tracks"]["x0"])
    sub = {k: v[: n // 5] for k, v in sc["tracks"].items()}
    oracle.set_num_threads(1)
    t0 = time.perf_counter()
    reps1, nb1 = 0, 0
    while time.perf_counter() - t0 < 3.0 or reps1 < 1:
        nb1 += len(M.bunches(sub, 7)["status"])
        reps1 += 1
    dt1 = time.perf_counter() - t0
    oracle.set_num_threads(cores)
    res["one_core"] = {"value": nb1 / dt1, "unit": UNIT, "cores": 1,
                       "sample": f"the first {n // 5} steps of that sample ({nb1 // reps1} "
                                 f"bunches), repeated {reps1} times, single-threaded"}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true",
                    help="device timing of regular launches only (no graph, FP64 leg, "
                         "end-to-end, other workloads or CPU legs)")
    ap.add_argument("--prec", choices=["fp32", "fp64"], default="fp32",
                    help="precision of the --quick timing")
    ap.add_argument("--launch", default=None,
                    help="block,ctas_per_sm instead of the autotuner's choice")
    ap.add_argument("--cap", type=int, default=None, help="records per telescope")
    ap.add_argument("--sweep", action="store_true", help="time a set of launch shapes")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["vertical_1tev", "inclined_20tev", "batched_256", "plain_fp64",
                             "adjoint_300gev"])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the workload's steps")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the other workloads, the adjoint and the generator legs")
    ap.add_argument("--leg", choices=["all", "generator", "adjoint", "fallback", "e2e_generated"],
                    default="all",
                    help="run one secondary leg alone (for profiling captures)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
    elif args.leg != "all":
        run_leg(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
