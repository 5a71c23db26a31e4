#!/usr/bin/env python
"""Throughput of the Cherenkov bunch hot path: bunches generated and
propagated per second.

Workload (default): one 1 TeV vertical gamma-like shower, 2e6 e+- steps,
19 telescope spheres, refraction tables 1000 x 64 up to 70 deg (seeded,
synthetic: see workloads/).  A step of the benchmark is one call of
cher_generate_propagate over all 2e6 steps: every bunch generated, refracted,
propagated, tested against the spheres and the crossings compacted.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank simulates its own shower (independent
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
                   "GPU in one persistent launch, 100 spheres over 2 x 2 km",
}
UNIT = "bunches/s"
WORKLOAD = "vertical_1tev"

# ---------------------------------------------------------------------------
# Algorithmic operation counts, from the algorithm as the oracle states it
# (each add, mul, fma, compare, select, convert, shift or logic op = 1; each
# sqrt, rsqrt or reciprocal = 1; implementation overhead excluded).  Per
# bunch, FP32/INT32 lane operations of the single-precision path, by stage;
# per emitting step, the FP64 operations of the yield.
# ---------------------------------------------------------------------------
OPS_PER_BUNCH_FP32 = {
    "sub_step_loop": 2,
    "philox4x32_10": 98,        # 10 x (2 mul.lo + 2 mul.hi + 4 xor) + 9 x 2 key adds
    "deviates": 9,              # 3 x (shift, convert, fma)
    "emission": 36,             # sub-step fraction, sin/cos of the azimuth, cone, lambda, height
    "rare_conditions": 3,
    "n_lookup_snell": 17,       # fine-table lookup, Snell ratio, sin^2, cos
    "tables": 24,               # two indices, two fractions, 2 x bilinear
    "ground_point_time": 21,    # sec, tan, offsets, X, Y, t, direction cosines
    "grid_and_sphere": 24,      # grid cell, one line-sphere test
    "output_counters": 8,       # amortised compaction and counters
}
OPS_PER_BUNCH = sum(OPS_PER_BUNCH_FP32.values())          # 242
# the floating-point part (everything but Philox), which the FP64 path runs
# on the FP64 pipe
FP64_OPS_PER_BUNCH = OPS_PER_BUNCH - OPS_PER_BUNCH_FP32["philox4x32_10"]
FP64_OPS_PER_STEP = 34          # yield chain: 24 mul/add + 1 division (~10 ops)
FP32_LANES_PER_SM = 128
FP64_FMA_PER_SM_CLK = 2         # GB300: 1/64 of the FP32 rate (ncu: 2 DFMA/cycle/SM)

# DRAM bytes (read + write) of one FP32 launch, from one ncu capture of the
# full-size vertical workload (128.21 MB read, 24.99 MB written, 128 threads
# x 8 CTAs per SM).  Reported only for that workload at full size and only
# while the kernel sources hash to what was profiled.
TRAFFIC = {"vertical_1tev": (153_202_688, "fcf7956156bb18a7")}
KERNEL_SOURCES = ("cher_kernels.cu", "cher_device.cuh", "cher_internal.h")


def _kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2006_14927_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(workload: str, scale: float):
    t = TRAFFIC.get(workload)
    if t is None or scale != 1.0 or _kernel_hash() != t[1]:
        return None
    return t[0]


# The same capture's pipe utilisation and issue activity (percent of peak),
# reported beside the operation counts under the same source-hash guard.
NCU_PIPES = {"alu": 41.0, "fma": 35.0, "fp64": 4.0, "issue_active": 73.3, "dram": 2.39}


def _ncu_pipes(workload: str, scale: float):
    return dict(NCU_PIPES) if _traffic(workload, scale) is not None else None


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


def run_reference(args):
    """The FP64 CPU oracle on a bounded sample of the same workload."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import oracle
    import workloads
    oracle.build()
    sample_steps = 20_000
    sc = workloads.vertical_1tev(n=sample_steps)
    M = oracle.Model(sc["atm"], sc["h_obs"], sc["telescopes"], t_ref=sc["t_ref"])
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
            "config": {"workload": f"{WORKLOAD} sample: first {sample_steps} of 2e6 steps",
                       "precision": "fp64 oracle (table variant)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample_steps} steps ({nb // args.steps} bunches) "
                                       f"of the 1 TeV vertical shower per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- workload (each rank its own shower: weak scaling) ----------------
    wl = args.workload
    if wl == "vertical_1tev":
        n_req = int(2_000_000 * args.scale)
        seed, track_base = shard(rank, n_req, 2)
        sc = workloads.vertical_1tev(n=n_req, seed=seed)
    elif wl == "inclined_20tev":
        n_req = int(100_000_000 * args.scale)
        seed, track_base = shard(rank, n_req, 5)
        sc = workloads.inclined_20tev(n=n_req, seed=seed)
    elif wl == "batched_256":
        n_req = int(200_000_000 * args.scale)
        seed, track_base = shard(rank, n_req, 3)
        sc = workloads.batched_256(total=n_req, seed=seed)
    else:
        sc = workloads.WORKLOADS[wl]()
        track_base = rank * len(sc["tracks"]["x0"])
    n = len(sc["tracks"]["x0"])
    t0 = time.perf_counter()
    ctx = P.Context(sc["atm"], sc["h_obs"], sc["telescopes"])
    ctx.build_refraction_tables(sc["H"], sc["Z"], sc["theta_max_deg"], sc["h_max"])
    table_s = time.perf_counter() - t0
    # records per telescope: the densest telescope of each workload fits
    # (batched: 12e6 x 100 telescopes x 40 B = 48 GB of the 288 GB)
    cap_full = {"vertical_1tev": 600_000, "batched_256": 12_000_000}.get(args.workload,
                                                                         8_000_000)
    cap = args.cap or (cap_full if args.workload == "vertical_1tev" else
                       max(200_000, int(cap_full * args.scale)))
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def measure(prec, steps, warmup, autotune, prof=None, reuse=None):
        if reuse is not None:
            dtr, out = reuse["dtr"], reuse["out"]
        else:
            dtr = P.device_tracks(sc["tracks"], prec, device=dev, t_ref=sc["t_ref"])
            out = ctx.alloc_hits(cap, prec, device=dev)
        pkw = {} if prof is None else dict(profile=prof[0], bin_gcm2=prof[1], axis_cos=prof[2])
        if autotune and args.launch is None:
            ctx.autotune(dtr, 11, prec, out)
        elif args.launch is not None:
            ctx.set_launch(*(int(v) for v in args.launch.split(",")))
        for _ in range(warmup):
            ctx.generate_propagate(dtr, 11, prec, out, track_base=track_base, **pkw)
        code, stats = ctx.sync_status(out)
        if code not in (0, 6):                      # 6: a buffer overflowed (counted)
            raise RuntimeError(f"status {code} in warm-up")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        barrier()
        w0 = time.perf_counter()
        for k in range(steps):
            flush.fill_(k & 0xff)                   # evict L2 between timed steps
            ev[k][0].record(stream)
            ctx.generate_propagate(dtr, 11, prec, out, track_base=track_base, **pkw)
            ev[k][1].record(stream)
        barrier()
        wall = time.perf_counter() - w0
        ms = [a.elapsed_time(b) for a, b in ev]
        code, stats = ctx.sync_status(out)
        return dict(ms=ms, wall=wall, stats=stats, dtr=dtr, out=out, code=code)

    steps, warmup = args.steps, args.warmup
    with ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
                      if os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0].isdigit()
                      else 0) as clk:
        r32 = measure(P.CHER_FP32_BULK, steps, warmup, autotune=True)
    clocks = clk.summary()
    launch = ctx.get_launch()
    if args.sweep and rank == 0:
        for shape in [(128, 1), (128, 2), (128, 4), (128, 6), (256, 1), (256, 2), (256, 3),
                      (256, 4), (512, 1), (512, 2), (128, 0), (256, 0)]:
            args.launch = f"{shape[0]},{shape[1]}"
            r = measure(P.CHER_FP32_BULK, 5, 2, autotune=False)
            t = statistics.median(r["ms"])
            print(json.dumps({"sweep": shape, "ms": t,
                              "bunches_per_s": float(r["stats"][3]) / (t / 1e3)}), flush=True)
        args.launch = f"{launch[0]},{launch[1]}"
        ctx.set_launch(*launch)
    if args.quick:
        t = sum(r32["ms"]) / 1e3
        if rank == 0:
            print(json.dumps({"quick": True, "value": float(r32["stats"][3]) * len(r32["ms"]) / t,
                              "unit": UNIT, "ms_per_step": 1e3 * t / len(r32["ms"]),
                              "launch": launch, "clocks": clocks}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    r64 = measure(P.CHER_FP64, max(3, steps // 4), max(3, min(warmup, 3)), autotune=False)
    # the longitudinal production profile (CERLDE) in the same launch:
    # 10 g/cm^2 bins to 2000 g/cm^2 of slant depth, one row per shower
    n_rows = max(len(sc["t_ref"]), 1)
    prof_t = torch.zeros((n_rows, 200), dtype=torch.float64, device=dev)
    axis_cos = np.cos(np.asarray(sc.get("axis_zenith_rad", np.zeros(n_rows)), float))
    r32p = measure(P.CHER_FP32_BULK, steps, max(3, min(warmup, 3)), autotune=False,
                   prof=(prof_t, 10.0, axis_cos), reuse=r32)
    # the atmospheric transmission draw (synthetic Rayleigh + aerosol table)
    ctx.set_transmission(workloads.synthetic_transmission(h_obs=sc["h_obs"], h_max=sc["h_max"]))
    r32t = measure(P.CHER_FP32_BULK, steps, max(3, min(warmup, 3)), autotune=False, reuse=r32)
    ctx.set_transmission(None)
    # the wavelength-dependent index (Edlen's dispersion of standard air, 9 nodes)
    ctx.set_dispersion(workloads.synthetic_dispersion(lambda1_nm=sc["lambda1_nm"],
                                                      lambda2_nm=sc["lambda2_nm"]))
    r32d = measure(P.CHER_FP32_BULK, steps, max(3, min(warmup, 3)), autotune=False, reuse=r32)
    ctx.set_dispersion(None)

    def total(r):
        return reduce_over_ranks(sum(r["ms"]) / 1e3, float(r["stats"][3]) * len(r["ms"]),
                                 world, dev)

    t32, b32 = total(r32)
    t64, b64 = total(r64)
    v32, v64 = b32 / t32, b64 / t64
    # the FP64 leg's device buffers are done with (the batched workload's
    # FP64 records alone take 86 GB)
    r64["out"] = r64["dtr"] = None
    torch.cuda.empty_cache()

    # ---- end to end: host buffers through the C ABI ---------------------
    e2e = None
    e2e_gen = None
    gen_leg = None
    if not args.no_e2e:
        prec = P.CHER_FP32_BULK
        host = {k: torch.as_tensor(np.ascontiguousarray(v)).pin_memory()
                for k, v in sc["tracks"].items() if k != "shower"}
        host["ux"], host["uy"], host["uz"] = (host[k].to(torch.float32).pin_memory()
                                              for k in ("ux", "uy", "uz"))
        host["shower"] = torch.as_tensor(
            np.ascontiguousarray(sc["tracks"]["shower"]).view(np.int32)).pin_memory()
        dtr = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
        dtr["t_ref"] = torch.as_tensor(sc["t_ref"], dtype=torch.float64, device=dev)
        out = r32["out"]
        n_tel = ctx.n_tel
        h_cnt = torch.empty(n_tel, dtype=torch.int64).pin_memory()
        h_st = torch.empty(P.NSTATS, dtype=torch.int64).pin_memory()
        # host records packed telescope after telescope: room for the FP32
        # leg's crossings (the same seed gives the same records every step;
        # the copies below refuse to truncate)
        n_rec = int(int(r32["stats"][9]) * 1.1) + 4096
        h_pos = torch.empty((n_rec, 4), dtype=torch.float32).pin_memory()
        h_tim = torch.empty((n_rec, 4), dtype=torch.float32).pin_memory()
        h_key = torch.empty(n_rec, dtype=torch.int64).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in host.values())

        # A three-stage pipeline over steps, every step still copying its whole
        # input up and its records back inside the timed region: step k+1's
        # inputs go up (copy stream) and step k-1's records come down (second
        # copy stream) while step k's kernel runs; two input sets, two output
        # buffers and two host record buffers.  Step k-1's download waits
        # until step k's kernel has started: a download already in flight when
        # the kernel's inputs landed held the kernel back until it ended
        # (seen on GB300 as kernel starts lined up with download ends).
        sets = [dtr, {k: torch.empty_like(v) for k, v in dtr.items()}]
        sets[1]["t_ref"].copy_(dtr["t_ref"])
        outs = [out, ctx.alloc_hits(cap, prec, device=dev)]
        hrec = [(h_pos, h_tim, h_key),
                (torch.empty_like(h_pos).pin_memory(), torch.empty_like(h_tim).pin_memory(),
                 torch.empty_like(h_key).pin_memory())]
        h_cnts = [h_cnt, torch.empty_like(h_cnt).pin_memory()]
        h_sts = [h_st, torch.empty_like(h_st).pin_memory()]
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
        barrier()
        e0 = time.perf_counter()
        d2h = run(steps)
        barrier()
        te = time.perf_counter() - e0
        te, _ = reduce_over_ranks(te, 0.0, world, dev)
        e2e = {"value": b32 / len(r32["ms"]) * steps / te, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "pipelined": "step k+1 up and step k-1 down during step k's kernel "
                            "(each download starts once the next kernel has)"}

        # end to end from shower parameters: the steps come from the device
        # generator (same shower, same step count), only the parameters and
        # its depth table go to the device
        if args.workload == "vertical_1tev" and world == 1:
            showers = [dict(e0_mev=1.0e6, zenith=0.0, azimuth=0.0, core_x=0.0, core_y=0.0,
                            n=int(len(sc["tracks"]["x0"])))]

            gen_buf = ctx.generate_steps(showers, 11, prec)

            def gen_step():
                dg = ctx.generate_steps(showers, 11, prec, out=gen_buf)
                ctx.generate_propagate(dg, 11, prec, out)
                ctx.pack_records(out, pk[0])
                h_cnt.copy_(out.count, non_blocking=True)
                h_st.copy_(out.stats, non_blocking=True)
                h_offs[0].copy_(pk[0]["offset"], non_blocking=True)
                torch.cuda.current_stream().synchronize()
                nbytes = (h_cnt.numel() + h_st.numel() + h_offs[0].numel()) * 8
                total = int(h_offs[0][-1])
                if total > n_rec:
                    raise RuntimeError("host record buffer too small")
                if total > 0:
                    h_pos[:total].copy_(pk[0]["pos"][:total], non_blocking=True)
                    h_tim[:total].copy_(pk[0]["tim"][:total], non_blocking=True)
                    h_key[:total].copy_(pk[0]["key"][:total], non_blocking=True)
                nbytes += total * 40
                torch.cuda.current_stream().synchronize()
                return nbytes, int(h_st[3])

            for _ in range(max(1, warmup // 2)):
                gen_step()
            g0 = time.perf_counter()
            gb = 0
            for _ in range(steps):
                gd2h, gbunch = gen_step()
                gb += gbunch
            tg = time.perf_counter() - g0
            # the generator alone (CUDA events around the whole call, whose
            # table upload blocks): 64 B of steps written per step
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
            g_gbs = showers[0]["n"] * 64 / (g_ms / 1e3) / 1e9
            gen_leg = {"ms_per_call": g_ms, "steps_per_s": showers[0]["n"] / (g_ms / 1e3),
                       "roofline": {"bound": "hbm", "achieved": g_gbs,
                                    "peak": float(peaks_.get("hbm_gbs", 6800.0)), "unit": "GB/s",
                                    "frac": g_gbs / float(peaks_.get("hbm_gbs", 6800.0)),
                                    "bytes_per_step": 64}}
            e2e_gen = {"value": gb / tg, "unit": UNIT,
                       "h2d_bytes_per_step": 64 + 16 + 4 * 1024 + 8,
                       "d2h_bytes_per_step": int(gd2h), "steps_generated": showers[0]["n"],
                       "bunches_per_step": gb // steps,
                       "note": "steps from cher_generate_steps (Philox draws, not the "
                               "host workload's)"}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (ALU bound) ----------------------
    peaks, src = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = sm_count * FP32_LANES_PER_SM * mhz * 1e6          # lane ops/s
    fp64_peak = sm_count * FP64_FMA_PER_SM_CLK * mhz * 1e6
    st = r32["stats"]
    bunches = float(st[3])
    emitting = float(st[1])
    per_launch_s = statistics.mean(r32["ms"]) / 1e3
    ops = bunches * OPS_PER_BUNCH
    achieved = ops / per_launch_s
    t_alu = ops / alu_peak
    t_fp64 = emitting * FP64_OPS_PER_STEP / fp64_peak
    cpu = cpu_baseline(args.workload) if world == 1 else None
    line = {
        "metric": METRIC, "value": v32, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": 1e3 * t32 / len(r32["ms"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT.get(args.workload, args.workload) +
                               (f" (scale {args.scale})" if args.scale != 1.0 else ""),
                   "steps_per_gpu": n, "n_showers": int(len(sc["t_ref"])),
                   "precision": "fp32_bulk (FP64 yield)", "bunches_per_step": int(bunches),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "launch": {"block": launch[0], "ctas_per_sm": launch[1],
                              "persistent": launch[1] > 0},
                   "table_build_s": table_s},
        "fp64": {"value": v64, "unit": UNIT, "ms_per_step": 1e3 * t64 / len(r64["ms"]),
                 "steps": len(r64["ms"]),
                 "roofline": {"bound": "fp64", "unit": "Tops/s",
                              "achieved": float(r64["stats"][3]) * FP64_OPS_PER_BUNCH /
                              (statistics.mean(r64["ms"]) / 1e3) / 1e12,
                              "peak": fp64_peak / 1e12,
                              "frac": float(r64["stats"][3]) * FP64_OPS_PER_BUNCH /
                              (statistics.mean(r64["ms"]) / 1e3) / fp64_peak,
                              "ops_per_bunch": FP64_OPS_PER_BUNCH,
                              "peak_source": f"{sm_count} SMs x {FP64_FMA_PER_SM_CLK} FP64 "
                                             f"lanes x {mhz:.0f} MHz"}},
        "fp32_over_fp64": v32 / v64,
        "transmission": {"ms_per_step": statistics.mean(r32t["ms"]),
                         "overhead": statistics.mean(r32t["ms"]) / statistics.mean(r32["ms"]) - 1,
                         "absorbed_frac": float(r32t["stats"][11]) / float(r32t["stats"][3]),
                         "table": "synthetic Rayleigh + aerosol, 16 x 121"},
        "dispersion": {"ms_per_step": statistics.mean(r32d["ms"]),
                       "overhead": statistics.mean(r32d["ms"]) / statistics.mean(r32["ms"]) - 1,
                       "value": float(r32d["stats"][3]) / (statistics.mean(r32d["ms"]) / 1e3),
                       "unit": UNIT, "bunches_per_step": int(r32d["stats"][3]),
                       "curve": "Edlen 1966 standard air, kappa = 1 at 400 nm, 9 nodes in "
                                "1/lambda"},
        "profile": {"ms_per_step": statistics.mean(r32p["ms"]),
                    "overhead": statistics.mean(r32p["ms"]) / statistics.mean(r32["ms"]) - 1.0,
                    "bins": int(prof_t.shape[1]), "bin_gcm2": 10.0, "rows": n_rows,
                    "depth": "slant" if np.any(axis_cos < 1.0) else "vertical"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": alu_peak / 1e12,
                     "unit": "Tops/s", "frac": achieved / alu_peak,
                     "traffic": _traffic(args.workload, args.scale),
                     "peak_source": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32/INT32 lanes x "
                                    f"{mhz:.0f} MHz ({src} max clock)",
                     "ops_per_bunch": OPS_PER_BUNCH,
                     "ops_by_stage": dict(OPS_PER_BUNCH_FP32),
                     "ncu_pct_of_peak": _ncu_pipes(args.workload, args.scale),
                     "roofline_ms": 1e3 * max(t_alu, t_fp64),
                     "fp64_yield_ms_at_peak": 1e3 * t_fp64,
                     "launch_ms": 1e3 * per_launch_s},
        "overflowed_records": int(r32["stats"][10]),
        "gpu_launches": len(r32["ms"]),
        "clocks": clocks,
        "e2e": e2e,
    }
    if e2e_gen is not None:
        line["e2e_generated"] = e2e_gen
        line["generator"] = gen_leg
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if args.workload == "vertical_1tev" and args.scale == 1.0 and world == 1:
        line["graph"] = graph_leg(ctx, r32, steps, flush, stream)
        line["adjoint"] = adjoint_leg(dev, steps)
        line["adjoint"]["cpu_baseline"] = cpu_baseline_readout()
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_leg(args):
    """One secondary leg alone: the step generator (2e6 steps of the 1 TeV
    vertical shower) or the adjoint (300 GeV shower, both precisions)."""
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


def graph_leg(ctx, r32, steps, flush, stream):
    """The same FP32 launch replayed from a captured CUDA graph (counter
    clears and the persistent kernel in one graph launch)."""
    import torch

    import paper_2006_14927_gb300 as P
    g = ctx.graph(r32["dtr"], 11, P.CHER_FP32_BULK, r32["out"])
    for _ in range(3):
        g.launch()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        g.launch()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    g.close()
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"ms_per_step": statistics.mean(ms),
            "value": float(r32["stats"][3]) / (statistics.mean(ms) / 1e3), "unit": UNIT}


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
    """The oracle as it stands on this host's cores, bounded sample: the
    workload's generator with its first 20 000 steps."""
    import oracle
    import workloads
    oracle.build()
    n = 20_000
    if workload == "batched_256":
        sc = workloads.batched_256(total=n)
    elif workload in ("plain_fp64", "adjoint_300gev"):
        sc = workloads.WORKLOADS[workload]()
        n = len(sc["tracks"]["x0"])
    else:
        sc = workloads.WORKLOADS[workload](n=n)
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
           "sample": f"{workload}: {n} steps ({nb // reps} bunches), repeated {reps} times, "
                     f"FP64 table variant, OpenMP over steps"}
    # the same single-threaded, on a fifth of the sample for about 3 s
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
                       "sample": f"{n // 5} steps ({nb1 // reps1} bunches), repeated {reps1} "
                                 f"times, single-threaded"}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true",
                    help="FP32 device timing only (no FP64, end-to-end or CPU legs)")
    ap.add_argument("--launch", default=None,
                    help="block,ctas_per_sm instead of the autotuner's choice")
    ap.add_argument("--cap", type=int, default=None, help="records per telescope")
    ap.add_argument("--sweep", action="store_true", help="time a set of launch shapes")
    ap.add_argument("--workload", default="vertical_1tev",
                    choices=["vertical_1tev", "inclined_20tev", "batched_256", "plain_fp64",
                             "adjoint_300gev"])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the workload's steps")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--leg", choices=["all", "generator", "adjoint", "fallback"], default="all",
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
