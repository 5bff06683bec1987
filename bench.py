"""Throughput of the Gaussian lattice Boltzmann hot path on GB300.

Default workload: plane Couette flow (Sec. 5.3) on the D2Q81 tensor-product
lattice (k = 3 summations, N = 4, 81 velocities), 512 x 256 nodes, walls moving
at -0.05 / +0.05, the three Knudsen numbers 0.01, 0.1, 1 stepped together as
three instances of one batched launch, FP32-deviation storage. A step is one
time step of all three instances (fused pull-stream + wall flux + BGK collide);
the populations (255 MB over both buffers) exceed the 129 MB L2, so no flush is
needed between steps. The same step is also timed in FP64 storage.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload couette|poiseuille|sod]

Under torchrun (N > 1) every rank runs its own copy of the workload (the
instances are independent: weak scaling, no data-path collective); rank 0
prints one JSON line with the whole-job throughput (max time over ranks).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "population updates/s and HBM GB/s (% peak), FP32 vs FP64 at <=1e-5 moment err"
UNIT = "pop-updates/s"


def workload(name):
    from paper_1905_04597_gb300 import inputs
    if name == "couette":
        c = inputs.COUETTE
        cfgs = [dict(dims=2, nx=c["nx"], ny=c["ny"], k=c["k"], kn=kn, u_wall_lo=c["u_wall_lo"],
                     u_wall_hi=c["u_wall_hi"]) for kn in c["kn"]]
        label = "couette_d2q81_512x256_kn{0.01,0.1,1}"
    elif name == "couette_4096":
        # the Couette workload on 4096 x 256: 2.0 GB per step, 16 times L2
        c = inputs.COUETTE
        cfgs = [dict(dims=2, nx=4096, ny=c["ny"], k=c["k"], kn=kn, u_wall_lo=c["u_wall_lo"],
                     u_wall_hi=c["u_wall_hi"]) for kn in c["kn"]]
        label = "couette_d2q81_4096x256_kn{0.01,0.1,1}"
    elif name == "couette_aniso":
        c = inputs.COUETTE_ANISO
        cfgs = [dict(dims=2, nx=c["nx"], ny=c["ny"], k=c["k"], x_level=c["x_level"], kn=kn,
                     u_wall_lo=c["u_wall_lo"], u_wall_hi=c["u_wall_hi"]) for kn in c["kn"]]
        label = "couette_d1q3xd1q17_1024x200_kn{0.01,0.1,1}"
    elif name in ("couette_zv", "couette_zv_xy"):
        c = inputs.COUETTE_ZV if name == "couette_zv" else inputs.COUETTE_ZV_XY
        cfgs = [dict(dims=2, nx=c["nx"], ny=c["ny"], k=c["k"], x_level=c["x_level"],
                     zv_axes=c["zv_axes"], kn=kn, u_wall_lo=c["u_wall_lo"],
                     u_wall_hi=c["u_wall_hi"]) for kn in c["kn"]]
        label = c["label"]
    elif name == "couette3d":
        c = inputs.COUETTE_3D
        cfgs = [dict(dims=3, nx=c["nx"], ny=c["ny"], nz=c["nz"], k=c["k"], kn=kn,
                     u_wall_lo=c["u_wall_lo"], u_wall_hi=c["u_wall_hi"]) for kn in c["kn"]]
        label = c["label"]
    elif name == "poiseuille":
        c = inputs.POISEUILLE
        cfgs = [dict(dims=2, nx=c["nx"], ny=c["ny"], k=c["k"], kn=kn, g=c["g"]) for kn in c["kn"]]
        label = "poiseuille_d2q289_1024x128_kn8"
    elif name == "batched":
        cfgs = [dict(dims=2, **r) for r in inputs.batched_instances(seed=0)]
        label = "batched_256_channels_k1-7_ny32-512_nx64"
    elif name == "sod":
        c = inputs.SOD
        cfgs = [dict(dims=1, nx=c["nx"], k=c["k"], kn=c["kn"])]
        label = "sod_d1q5_1000"
    else:
        raise SystemExit(f"unknown workload {name}")
    return cfgs, label


def lattice_axes(cfg):
    """(N, NX, Q1y, Q1x, zv) of a 2D workload instance: levels along y and x,
    velocities per axis and the mask of axes on the 2N+2 hierarchy."""
    N = cfg["k"] + 1
    NX = cfg.get("x_level") or N
    zv = cfg.get("zv_axes", 0)
    return N, NX, 2 * N + 1 + (1 if zv & 2 else 0), 2 * NX + 1 + (1 if zv & 1 else 0), zv


def workload_config(name, args, world):
    """The `config` object of both arms' lines for a workload of workload():
    what the workload is and how it is laid out and timed, nothing that
    depends on the arm (the arm's storage and kernel choices are reported
    beside it)."""
    cfgs, label = workload(name)
    c = cfgs[0]
    dims = c["dims"]
    N, NX, Q1y, Q1x, _ = lattice_axes(c)
    Q = Q1y * Q1x if dims == 2 else ((2 * N + 1) ** 3 if dims == 3 else 2 * N + 1)
    nodes = c["nx"] * (c["ny"] if dims >= 2 else 1) * (c["nz"] if dims == 3 else 1)
    pops = Q * nodes * len(cfgs)
    return {"workload": label, "lattice": f"D{dims}Q{Q}", "k": N - 1, "nodes": nodes,
            "instances": len(cfgs),
            "l2": (f"FP32 populations {4 * pops / 1e6:.0f} MB per buffer, two buffers "
                   f"{8 * pops / 1e6:.0f} MB " + ("> 129 MB L2" if 8 * pops > 129e6 else
                                                   "(fit in the 129 MB L2)") + "; no flush"),
            "parallelism": f"instances batched per launch; {world} rank(s), independent copies",
            "tiles": args.tiles}


KERNEL_SOURCES = ("glbm_device.cuh", "glbm_step2d.cuh", "glbm_step2d_pair.cuh",
                  "glbm_step2d_launch.cuh", "glbm_tiles.h", "glbm_internal.h")
KERNEL_SOURCES_3D = KERNEL_SOURCES + ("glbm_step3d.cuh", "glbm_step3d.cu")


def kernel_source_hash(kernel=""):
    """SHA-256 (first 16 hex digits) of the sources of the fused 2D step, and
    of the 3D step's own sources too for a k_step3d kernel."""
    import hashlib
    h = hashlib.sha256()
    for f in (KERNEL_SOURCES_3D if kernel.startswith("k_step3d") else KERNEL_SOURCES):
        with open(os.path.join(ROOT, "paper_1905_04597_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    capture (profiles/traffic.json), or None when there is none for the kernel
    sources as they are now."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    for r in rec.get("captures", []):
        if (r.get("kernel") == kernel and r.get("workload") == workload
                and r.get("source_hash") == kernel_source_hash(kernel)):
            return r["dram_bytes_per_launch"]
    return None


def fp64_pipe_record(kernel, workload):
    """FP64 instructions per launch of `kernel` on `workload` from the committed
    ncu counters (profiles/traffic.json), or None if they do not describe the
    current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    for r in rec.get("fp64", []):
        if (r.get("kernel") == kernel and r.get("workload") == workload
                and r.get("source_hash") == kernel_source_hash()):
            return r
    return None


FP64_INST_PER_SM_CLK = 2  # FP64 pipe issue rate of a GB300 SM (ncu peak_sustained of DFMA)
N_SM = 152


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler runs (its first sample is
            # in), so that nvidia-smi's own start-up does not overlap it
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
            time.sleep(0.05)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 alone)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x):
    """The largest x over the ranks of the initialised process group (x alone
    without one): the job's time is that of its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms_max):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (weak scaling: each rank runs its own copy of the workload)."""
    return units_per_rank * world / (ms_max / 1e3)


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build_library()
    if world > 1:
        torch.distributed.barrier()
    from paper_1905_04597_gb300 import glbm

    if args.workload == "couette_slab":
        with ClockSampler(local) as clk:
            res = measure_slab(args.steps, args.warmup, rank, world)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": res["pop_updates_per_s"], "unit": UNIT,
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                              "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                              "data": "synthetic",
                              "config": {"workload": res["label"],
                                         "parallelism": f"x slabs over {world} rank(s), halo "
                                                        f"exchange every {res['steps_per_exchange']} "
                                                        f"steps",
                                         "l2": "2.0 GB of populations per buffer set; no flush"},
                              "slab": res, "clocks": clk.summary(),
                              "gpu_launches": res["launches"]}), flush=True)
        return
    if args.workload == "batched":
        with ClockSampler(local) as clk:
            res = measure_batched(steps32=args.steps, steps64=max(args.steps // 8, 8),
                                  warmup=args.warmup, autotune=args.tiles == "autotune",
                                  rank=rank, world=world)
        if rank == 0:
            b = res["fp32_batched"]
            cpu = cpu_baseline_batched() if not args.no_cpu_baseline and world == 1 else None
            print(json.dumps({"metric": METRIC, "value": b["pop_updates_per_s"], "unit": UNIT,
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": b["ms_per_step"], "higher_is_better": True,
                              "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                              "data": "synthetic",
                              "config": {"workload": "batched_256_channels_k1-7_ny32-512_nx64",
                                         "parallelism": f"the 256 instances split by population "
                                                        f"bytes over {world} rank(s), no "
                                                        f"data-path collective",
                                         "l2": "2.6 GB of populations per buffer set; no flush"},
                              "batched": res, "clocks": clk.summary(), "cpu_baseline": cpu,
                              "gpu_launches": int(round(b["launches_per_step"] * args.steps))}),
                  flush=True)
        return
    if args.workload == "adjoint":
        with ClockSampler(local) as clk:
            res = measure_adjoint(reps=max(1, args.steps // 4000), warmup_steps=args.warmup)
        if rank == 0:
            cpu = (cpu_baseline_adjoint(args.cpu_seconds)
                   if not args.no_cpu_baseline and world == 1 else None)
            print(json.dumps({"metric": METRIC, "value": res["pop_steps_per_s"], "unit": UNIT,
                              "n_gpus": world, "steps": res["steps"], "warmup": args.warmup,
                              "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                              "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                              "data": "synthetic", "config": {"workload": res["label"]},
                              "roofline": res["roofline"], "adjoint": res, "clocks": clk.summary(),
                              "cpu_baseline": cpu, "gpu_launches": res["launches"]}), flush=True)
        return
    cfgs, label = workload(args.workload)
    dims = cfgs[0]["dims"]
    N, NX, Q1y, Q1x, ZV = lattice_axes(cfgs[0])
    Q = Q1y * Q1x if dims == 2 else ((2 * N + 1) ** 3 if dims == 3 else 2 * N + 1)
    nodes = cfgs[0]["nx"] * (cfgs[0]["ny"] if dims >= 2 else 1) * (cfgs[0]["nz"] if dims == 3 else 1)
    n_inst = len(cfgs)
    pops_per_step = Q * nodes * n_inst
    stream = torch.cuda.current_stream()

    tiles_used = {}

    def kernel_name(prec, lat):
        """Name of the step kernel the context runs, with every template
        argument (the form profiles/traffic.json records)."""
        G, R, V = lat.tile_shape(N - 1)
        t = "float" if prec == glbm.FP32_DEV else "double"
        if dims == 3:
            return f"k_step3d<{N},{t},{G},{R}>"
        zy, zx = (1 if ZV & 2 else 0), (1 if ZV & 1 else 0)
        if V == 2:
            return f"k_step2d_pair<{N},{G},{R},{NX},{zy},{zx}>"
        return f"k_step2d<{N},{t},{G},{R},{NX},{zy},{zx}>"

    def choose_tiles(lat, prec):
        """Autotune, keep the defaults, or (idx:<i>) take candidate i of the
        FP32 list for the workload's level (FP64 keeps its default)."""
        if args.tiles == "autotune":
            lat.autotune(reps=10)
        elif args.tiles.startswith("idx:") and prec == glbm.FP32_DEV:
            t = [-1] * glbm.LEVELS
            t[N - 1] = int(args.tiles[4:])
            lat.set_tiles(t)

    wall_mode = {}

    def timed(prec, steps, warmup):
        lat = glbm.Lattice([dict(c, prec=prec) for c in cfgs])
        if dims >= 2:
            choose_tiles(lat, prec)
            tiles_used[prec] = kernel_name(prec, lat)
            wall_mode[prec] = lat.wall_launch if dims == 2 else -1
        lat.step(warmup)
        lat.sync()
        l0 = lat.kernel_launches
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(stream)
            lat.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = lat.kernel_launches - l0
        lat.sync()
        lat.close()
        ms = max_over_ranks(ms)
        return ms, launches, clk.summary()

    steps, warmup = args.steps, args.warmup
    if args.only:
        # one precision's timed steps alone (what a profiler capture needs)
        prec = glbm.FP32_DEV if args.only == "fp32" else glbm.FP64
        ms, launches, clk = timed(prec, steps, warmup)
        if rank == 0:
            s = 4 if prec == glbm.FP32_DEV else 8
            print(json.dumps({"metric": METRIC, "value": job_throughput(pops_per_step * steps,
                                                                        world, ms),
                              "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
                              "ms_per_step": ms / steps, "higher_is_better": True,
                              "scaling": "weak", "vs_baseline": None,
                              "dtype": "f32" if s == 4 else "f64", "data": "synthetic",
                              "config": {"workload": label, "only": args.only,
                                         "tiles": args.tiles},
                              "kernel": tiles_used.get(prec),
                              "hbm_gbs_algorithmic": 2 * s * pops_per_step / (ms / steps / 1e3) / 1e9,
                              "clocks": clk, "gpu_launches": launches}), flush=True)
        return
    ms32, launches, clocks = timed(glbm.FP32_DEV, steps, warmup)
    ms64, _, clocks64 = timed(glbm.FP64, max(steps // 4, 4), warmup)
    steps64 = max(steps // 4, 4)

    value = job_throughput(pops_per_step * steps, world, ms32)
    value64 = job_throughput(pops_per_step * steps64, world, ms64)
    peak, peak_kind = peaks()
    bytes32 = 2 * 4 * pops_per_step       # algorithmic bytes of one launch (read + write)
    bytes64 = 2 * 8 * pops_per_step
    per_launch_ms = ms32 / steps
    gbs32 = bytes32 / (per_launch_ms / 1e3) / 1e9
    gbs64 = bytes64 / (ms64 / steps64 / 1e3) / 1e9

    # end to end through the public API with pinned host buffers: upload the initial
    # fields, run a chunk of steps, read every moment back
    e2e = None
    if dims >= 2:
        lb_per_call = 100
        lat = glbm.Lattice([dict(c, prec=glbm.FP32_DEV) for c in cfgs])
        choose_tiles(lat, glbm.FP32_DEV)
        shp = lat.shape(0)
        nf = 9 if dims == 3 else 7
        pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
        rho = pin(np.ones(shp))
        ux = pin(np.zeros(shp))
        uy = pin(np.zeros(shp))
        outs = [torch.empty((nf,) + shp, dtype=torch.float64).pin_memory() for _ in cfgs]
        reps = max(2, min(20, steps // lb_per_call))

        def one():
            for i in range(n_inst):
                lat.set_equilibrium(i, rho, ux, uy)
            lat.step(lb_per_call)
            for i in range(n_inst):
                lat.moments(i, out=outs[i])

        one()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            one()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        lat.close()
        e2e = {"value": pops_per_step * lb_per_call * world / dt, "unit": UNIT,
               "h2d_bytes_per_step": 3 * 8 * nodes * n_inst,
               "d2h_bytes_per_step": nf * 8 * nodes * n_inst,
               "lb_steps_per_step": lb_per_call,
               "call": "glbm_set_equilibrium(host) x3 + glbm_step(100) + glbm_moments(host) x3"}

    precision = (precision_check(cfgs, precision_steps(args.workload))
                 if dims >= 2 and not args.no_precision else None)
    # FP64 is bound by the FP64 pipe: its instructions per launch come from the
    # committed ncu counters, the peak from the library's FMA-throughput probe
    # (measured here; the pipe's nominal rate times the clock beside it)
    fp64_roof = None
    rec = fp64_pipe_record(tiles_used.get(glbm.FP64), label)
    if rec is not None:
        ach = rec["dp_inst_per_launch"] / (ms64 / steps64 / 1e3) / 1e9
        pk = glbm.measure_fp64_rate() / 1e9
        nominal = (FP64_INST_PER_SM_CLK * N_SM * clocks64["sm_max_mhz"] / 1e3
                   if clocks64.get("sm_max_mhz") else None)
        fp64_roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "G FP64 inst/s",
                     "peak_kind": "measured (glbm_measure_fp64_rate: independent DFMA chains)",
                     "peak_nominal": nominal, "frac": ach / pk, "hbm_frac": gbs64 / peak,
                     "dp_flops_per_pop": rec["dp_flops_per_launch"] / pops_per_step}
    batched = (measure_batched(autotune=args.tiles == "autotune", rank=rank, world=world)
               if (args.workload == "couette" and not args.no_batched) else None)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, budget_s=args.cpu_seconds)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms32 / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.workload, args, world),
        "storage": "fp32 deviations",
        "wall_densities": {1: "own launch", 0: "in the tiles"}.get(
            wall_mode.get(glbm.FP32_DEV, -1), "no walls"),
        "mlups": nodes * n_inst * steps * world / (ms32 / 1e3) / 1e6,
        "hbm_gbs_algorithmic": gbs32,
        "fp64": {"value": value64, "unit": UNIT, "ms_per_step": ms64 / steps64, "steps": steps64,
                 "kernel": tiles_used.get(glbm.FP64, "k_step1d"), "roofline": fp64_roof,
                 "hbm_gbs_algorithmic": gbs64, "frac_of_hbm": gbs64 / peak,
                 "clocks": clocks64},
        "roofline": {"bound": "hbm", "achieved": gbs32, "peak": peak, "unit": "GB/s",
                     "frac": gbs32 / peak,
                     "traffic": measured_traffic(tiles_used.get(glbm.FP32_DEV), label),
                     "kernel": tiles_used.get(glbm.FP32_DEV, "k_step1d"),
                     "bytes_per_launch": bytes32, "peak_source": peak_kind,
                     "launches_per_step": launches / steps,
                     "timing": "CUDA events over the timed steps; a step's every launch (the "
                               "wall-density launch too, where the step has one) is counted "
                               "against the step kernel"},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "precision": precision,
        "batched": batched,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


STEPS_PER_SOLVE = 2000  # a channel solve of the batched workload


def precision_steps(name):
    """Step count at which a workload's FP32 accuracy is stated: the Couette
    workload's 20000 steps, the Poiseuille workload's 2000, else 2000."""
    from paper_1905_04597_gb300 import inputs
    return {"couette": inputs.COUETTE["steps"],
            "poiseuille": inputs.POISEUILLE["steps"]}.get(name, 2000)


def precision_check(cfgs, steps):
    """FP32-deviation against FP64 storage on the GPU, every instance of the
    workload (one per Knudsen number) stepped together from the same initial
    state for `steps` steps; the FP64 path matches the CPU oracle to 1e-12 in
    the parity tests. Per instance and field: the error metric of the parity
    tests (max |got - want| over the field's max, floored at 1e-3 of the
    per-node sum of the moment's absolute terms) and the plain field max-norm
    error without the floor. Runs outside the timed region."""
    from paper_1905_04597_gb300 import glbm, metrics
    t0 = time.perf_counter()
    runs = {}
    for prec in (glbm.FP32_DEV, glbm.FP64):
        lat = glbm.Lattice([dict(c, prec=prec) for c in cfgs])
        lat.step(steps)
        lat.sync()
        runs[prec] = [(lat.moments(i), lat.get_populations(i) if prec == glbm.FP64 else None)
                      for i in range(len(cfgs))]
        lat.close()
    dims = cfgs[0]["dims"]
    names = (metrics.FIELDS_3D if dims == 3 else
             (metrics.FIELDS_2D if dims == 2 else metrics.FIELDS_1D))
    q1x, zv = ((lattice_axes(cfgs[0])[3], cfgs[0].get("zv_axes", 0)) if dims == 2
               else (None, 0))
    per, worst = [], (0.0, None, None)
    for i, cfg in enumerate(cfgs):
        got, (ref, F) = runs[glbm.FP32_DEV][i][0], runs[glbm.FP64][i]
        want = np.stack([ref[n] for n in names])
        errs = metrics.rel_errors(got, want, dims=dims, F=F, q1x=q1x, zv=zv)
        plain = metrics.plain_errors(got, want, dims=dims)
        per.append({"kn": cfg.get("kn"), "rel_err": errs, "plain_rel_err": plain,
                    "ref_max_abs": {n: float(np.abs(ref[n]).max()) for n in names}})
        for n, e in errs.items():
            if e > worst[0]:
                worst = (e, cfg.get("kn"), n)
    return {"steps": steps,
            "reference": "FP64 storage on the GPU (equal to the CPU oracle to 1e-12 in the tests)",
            "instance": {k: cfgs[0][k] for k in ("k", "x_level", "zv_axes", "nx", "ny", "nz")
                         if k in cfgs[0]},
            "per_kn": per, "max": worst[0], "worst": {"kn": worst[1], "field": worst[2]},
            "plain_qx_max": max((p["plain_rel_err"]["qx"] or 0.0) for p in per),
            "seconds": time.perf_counter() - t0}


ADJ_BYTES_PER_POP = 36  # per population and time step: see measure_adjoint


def measure_adjoint(reps=1, warmup_steps=200):
    """Throughput of the flow-rate gradient (glbm_adjoint_flowrate) on the adjoint
    workload (D2Q121 256 x 128, Kn 0.1, g 1e-6, FP32 forward, 4000 steps,
    checkpoints every 100). Per population and time step the algorithmic
    traffic is 36 bytes: the forward step reads and writes the FP32 state
    (8 B), the segment recomputed from its checkpoint does it again (8 B), and
    the adjoint step reads the forward state (4 B) and the FP64 adjoint state
    of the next step (8 B) and writes the adjoint state (8 B)."""
    import torch
    from paper_1905_04597_gb300 import glbm, inputs
    c = inputs.ADJOINT
    cfg = dict(dims=2, nx=c["nx"], ny=c["ny"], k=c["k"], kn=c["kn"], g=c["g"], prec=glbm.FP32_DEV)
    Q = (2 * c["k"] + 3) ** 2
    pops = Q * c["nx"] * c["ny"]
    lat = glbm.Lattice(cfg)
    lat.adjoint_flowrate(warmup_steps, c["ckpt_every"])  # warm-up (graphs, buffers)
    torch.cuda.synchronize()
    l0 = lat.kernel_launches
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        for _ in range(reps):
            J, dtau, dg = lat.adjoint_flowrate(c["steps"], c["ckpt_every"])
        dt = time.perf_counter() - t0
    launches = lat.kernel_launches - l0
    lat.close()
    steps = c["steps"] * reps
    peak, peak_kind = peaks()
    gbs = ADJ_BYTES_PER_POP * pops * steps / dt / 1e9
    return {"label": f"adjoint_d2q{Q}_{c['nx']}x{c['ny']}_kn{c['kn']}_{c['steps']}steps_ckpt{c['ckpt_every']}",
            "steps": steps, "ms_per_step": dt / steps * 1e3, "pop_steps_per_s": pops * steps / dt,
            "solves_per_s": reps / dt, "J": float(J[0]), "dJ_dtau": float(dtau[0]),
            "dJ_dg": float(dg[0]), "launches": int(launches),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "traffic": None, "peak_source": peak_kind,
                         "bytes_per_pop_step": ADJ_BYTES_PER_POP,
                         "timing": "host wall clock around the synchronous call (forward, "
                                   "checkpoints, recomputed segments and adjoint sweep)"},
            "clocks": clk.summary()}


def measure_slab(steps, warmup, rank=0, world=1):
    """One Couette D2Q81 lattice of 4096 x 256 (Kn 0.1, walls at -+0.05, FP32)
    split into x slabs over the ranks (slab.SlabLattice, autotuned): each rank
    steps its Ls = 4096 / world owned columns plus H = m x 4 halo columns per
    side, and the halos are exchanged once every m steps (deep halos, m from
    slab.default_depth; NCCL between GPUs, one rank copies its own columns
    across). The value counts the undivided lattice's population updates over
    the slowest rank's time (strong scaling)."""
    import torch
    from paper_1905_04597_gb300 import glbm, slab
    cfg = dict(dims=2, nx=4096, ny=256, k=3, kn=0.1, u_wall_lo=-0.05, u_wall_hi=0.05,
               prec=glbm.FP32_DEV)
    s = slab.SlabLattice(cfg, rank, world)
    shp = (cfg["ny"], cfg["nx"])
    s.set_equilibrium_global(np.ones(shp), np.zeros(shp), np.zeros(shp))
    s.lat.autotune(reps=5)
    s.advance(warmup)
    l0 = s.lat.kernel_launches
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.advance(steps)
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    launches = s.lat.kernel_launches - l0
    pops = 81 * cfg["nx"] * cfg["ny"]
    halo = 2 * 81 * cfg["ny"] * s.H * 4  # bytes each rank sends per exchange (both sides)
    out = {"label": "couette_slab_d2q81_4096x256_kn0.1", "ranks": world, "owned_columns": s.Ls,
           "halo_columns_per_side": s.H, "steps_per_exchange": s.depth,
           "halo_bytes_sent_per_rank_exchange": halo,
           "halo_bytes_sent_per_rank_step": halo / s.depth,
           "step_bytes_per_rank": 8 * 81 * cfg["ny"] * (s.Ls + 2 * s.H),
           "redundant_fraction": 2 * s.H / s.Ls,
           "tiles": s.lat.tiles()[3], "dataflow": s.lat.dataflow,
           "ms_per_step": ms / steps, "pop_updates_per_s": pops * steps / (ms / 1e3),
           "launches": launches}
    s.lat.close()
    return out


def batch_share(rank, world):
    """This rank's instances of the 256-channel batch: the batch split across
    the ranks by population bytes (shard.partition_by_bytes), with the split's
    balance."""
    from paper_1905_04597_gb300 import inputs, shard
    recipe = inputs.batched_instances(seed=0)
    sizes = [shard.instance_bytes(r) for r in recipe]
    parts = shard.partition_by_bytes(sizes, world)
    loads = [sum(sizes[i] for i in p) for p in parts]
    return ([recipe[i] for i in parts[rank]], recipe,
            {"instances": len(parts[rank]), "bytes": loads[rank], "index": parts[rank],
             "max_share_over_mean": max(loads) * world / sum(loads)})


def measure_batched(steps32=256, steps64=64, warmup=8, autotune=True, rank=0, world=1):
    """Solves/s of the 256-instance heterogeneous batch in FP32 (one launch per
    level present per step) against the same instances in FP64, one context
    (and one launch per step) per instance. With several ranks each steps its
    byte-balanced share of the batch (no data-path collective), and the batch's
    time is the slowest rank's (strong scaling: the batch is fixed)."""
    import torch
    from paper_1905_04597_gb300 import glbm
    recipe, recipe_all, share = batch_share(rank, world)

    def pops_of(rs):
        return sum((2 * r["k"] + 3) ** 2 * r["nx"] * r["ny"] for r in rs)

    pops = pops_of(recipe_all)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def barrier():
        import torch.distributed as dist
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    lat = glbm.Lattice([dict(dims=2, prec=glbm.FP32_DEV, **r) for r in recipe], hetero=True)
    if autotune:
        lat.autotune(reps=5)
    tiles = lat.tiles()
    lat.step(warmup)
    lat.sync()
    l0 = lat.kernel_launches
    barrier()
    e0.record(stream)
    lat.step(steps32)
    e1.record(stream)
    barrier()
    ms32 = max_over_ranks(e0.elapsed_time(e1))
    launches32 = lat.kernel_launches - l0
    # the final gather: every instance's flow rate J (channel diagnostics), in
    # batch order on every rank (outside the timed region)
    mine = {idx: lat.channel_diagnostics(k)[1]["flow_rate"] for k, idx in enumerate(share["index"])}
    if world > 1:
        import torch.distributed as dist
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        for p in parts:
            mine.update(p)
    flow = [mine[i] for i in range(len(recipe_all))]
    lat.close()
    singles = [glbm.Lattice(dict(dims=2, prec=glbm.FP64, **r)) for r in recipe]
    for x in singles:
        x.step(2)
    barrier()
    e0.record(stream)
    for x in singles:
        x.step(steps64)
    e1.record(stream)
    barrier()
    ms64 = max_over_ranks(e0.elapsed_time(e1))
    for x in singles:
        x.close()
    sps32 = steps32 / (ms32 / 1e3)          # steps/s of the whole batch
    sps64 = steps64 / (ms64 / 1e3)
    n = len(recipe_all)
    share = {k: v for k, v in share.items() if k != "index"}
    return {"instances": n, "pop_updates_per_step": pops, "ranks": world, "rank0_share": share,
            "gathered_flow_rates": {"instances": len(flow), "sum": float(np.sum(flow)),
                                    "finite": bool(np.all(np.isfinite(flow)))},
            "fp32_batched": {"solves_per_s": n * sps32 / STEPS_PER_SOLVE, "tiles": tiles,
                             "pop_updates_per_s": pops * sps32, "ms_per_step": ms32 / steps32,
                             "launches_per_step": launches32 / steps32},
            "fp64_one_instance_per_launch": {"solves_per_s": n * sps64 / STEPS_PER_SOLVE,
                                             "pop_updates_per_s": pops * sps64,
                                             "ms_per_step": ms64 / steps64,
                                             "launches_per_step": len(recipe)},
            "speedup": sps32 / sps64, "steps_per_solve": STEPS_PER_SOLVE}


def _omp_threads():
    """Threads an -fopenmp oracle uses here (OMP_NUM_THREADS, else every core)."""
    try:
        return max(1, int(os.environ.get("OMP_NUM_THREADS", "")))
    except ValueError:
        return os.cpu_count() or 1


def _host_cpu():
    """This host's CPU model and logical core count (lscpu when present)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model or "unknown", "nproc": os.cpu_count()}


def _oracle_sample(name, openmp):
    """(oracle lattice, initial state, populations per step, label, first instance)
    for one instance of the workload, on the single-thread or the -fopenmp build."""
    from oracle import oracle as orc
    cfgs, label = workload(name)
    c = cfgs[0]
    N = c["k"] + 1
    dims = c["dims"]
    if dims == 2:
        _, NX, Q1y, Q1x, zv = lattice_axes(c)
        o = orc.Lattice(2, NX, N, c["nx"], c["ny"], orc.BC_WALLS,
                        orc.tau_from_kn(N, c["ny"], c["kn"], zv=zv & 2), c.get("u_wall_lo", 0.0),
                        c.get("u_wall_hi", 0.0), c.get("g", 0.0), zv=zv, openmp=openmp)
        X = o.equilibrium(np.ones((c["ny"], c["nx"])), np.zeros((c["ny"], c["nx"])),
                          np.zeros((c["ny"], c["nx"])))
        pops = Q1y * Q1x * c["nx"] * c["ny"]
    elif dims == 3:
        o = orc.Lattice(3, N, N, c["nx"], c["ny"], orc.BC_WALLS, orc.tau_from_kn(N, c["ny"], c["kn"]),
                        c.get("u_wall_lo", 0.0), c.get("u_wall_hi", 0.0), c.get("g", 0.0),
                        NZ=N, Lz=c["nz"], openmp=openmp)
        shp = (c["nz"], c["ny"], c["nx"])
        X = o.equilibrium(np.ones(shp), np.zeros(shp), np.zeros(shp), np.zeros(shp))
        pops = (2 * N + 1) ** 3 * c["nx"] * c["ny"] * c["nz"]
    else:
        o = orc.Lattice(1, N, 0, c["nx"], 1, orc.BC_BOUNCEBACK,
                        orc.tau_from_kn(N, c["nx"], c["kn"]), openmp=openmp)
        X = o.equilibrium(np.ones(c["nx"]), np.zeros(c["nx"]))
        pops = (2 * N + 1) * c["nx"]
    return o, X, pops, label, c


def cpu_baseline(name, budget_s=15.0, steps=None):
    """The FP64 oracle, as it stands, on this host's cores over a bounded sample
    of the workload (the full lattice of one instance for as many steps as fit
    half the budget, at least one): once on all cores (its -fopenmp build,
    whose collision runs over rows in parallel with identical results; this is
    the reported value) and once single-threaded."""
    out = {}
    for openmp in (True, False):
        o, X, pops, label, c = _oracle_sample(name, openmp)
        t0 = time.perf_counter()
        X, _ = o.run(X, 1)
        one = time.perf_counter() - t0
        n = steps or max(1, int(0.5 * budget_s / max(one, 1e-6)) - 1)
        t0 = time.perf_counter()
        X, _ = o.run(X, n)
        dt = time.perf_counter() - t0
        out[openmp] = (pops * n / dt, n, dt, label, c)
    v, n, dt, label, c = out[True]
    v1, n1, dt1 = out[False][:3]
    cores = _omp_threads()
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "host": _host_cpu(),
            "sample": f"{label}: one instance (Kn {c['kn']}), full lattice, {n} steps, FP64, "
                      f"{cores} threads (collision over rows), {dt:.1f} s",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"the same lattice, {n1} steps, {dt1:.1f} s"}}


def cpu_baseline_batched():
    """The FP64 oracle over one step of every instance of the 256-channel batch
    (about 0.65 G population updates), on all cores and single-threaded: a
    sample with the batch's own mix of levels, sizes and boundary kinds."""
    from oracle import oracle as orc
    cfgs, label = workload("batched")
    out = {}
    for openmp in (True, False):
        pops, dt = 0, 0.0
        for c in cfgs:
            N = c["k"] + 1
            o = orc.Lattice(2, N, N, c["nx"], c["ny"], orc.BC_WALLS,
                            orc.tau_from_kn(N, c["ny"], c["kn"]), c["u_wall_lo"], c["u_wall_hi"],
                            c["g"], openmp=openmp)
            shp = (c["ny"], c["nx"])
            X = o.equilibrium(np.ones(shp), np.zeros(shp), np.zeros(shp))
            t0 = time.perf_counter()
            o.run(X, 1)
            dt += time.perf_counter() - t0
            pops += (2 * N + 1) ** 2 * c["nx"] * c["ny"]
        out[openmp] = (pops / dt, dt)
    cores = _omp_threads()
    return {"value": out[True][0], "unit": UNIT, "cores": cores, "kind": "oracle",
            "host": _host_cpu(),
            "sample": f"{label}: one step of each of the {len(cfgs)} instances, FP64, {cores} "
                      f"threads (collision over rows), {out[True][1]:.1f} s",
            "single_thread": {"value": out[False][0], "unit": UNIT, "cores": 1,
                              "sample": f"the same, {out[False][1]:.1f} s"}}


def cpu_baseline_adjoint(budget_s=15.0):
    """The oracle's gradient of the flow rate (forward-mode dual numbers: the
    state and its tau and g tangents in one pass, single-threaded) on the
    adjoint workload's lattice, for as many steps from rest as fit about the
    budget; per population and time step, as the GPU figure counts."""
    from oracle import oracle as orc
    from paper_1905_04597_gb300 import inputs
    c = inputs.ADJOINT
    N = c["k"] + 1
    o = orc.Lattice(2, N, N, c["nx"], c["ny"], orc.BC_WALLS, orc.tau_from_kn(N, c["ny"], c["kn"]),
                    0.0, 0.0, c["g"])
    shp = (c["ny"], c["nx"])
    X = o.equilibrium(np.ones(shp), np.zeros(shp), np.zeros(shp))
    t0 = time.perf_counter()
    o.flowrate_grad(X, 1)
    one = time.perf_counter() - t0
    n = max(1, int(budget_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    o.flowrate_grad(X, n)
    dt = time.perf_counter() - t0
    pops = (2 * N + 1) ** 2 * c["nx"] * c["ny"]
    return {"value": pops * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host": _host_cpu(),
            "sample": f"D2Q{(2 * N + 1) ** 2} {c['nx']}x{c['ny']}, Kn {c['kn']}: J and its tau "
                      f"and g derivatives by dual numbers over {n} steps, FP64, one thread, "
                      f"{dt:.1f} s"}


def run_reference(args):
    """The oracle timed as the reference arm, on all cores (its -fopenmp build):
    each step one oracle time step of a bounded slab of the workload (a column
    strip of the lattice)."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.build_openmp()
    cfgs, label = workload(args.workload)
    c = cfgs[0]
    N = c["k"] + 1
    dims = c["dims"]
    budget = 120.0
    total_steps = args.steps + args.warmup
    if dims == 2:
        ny = c["ny"]
        _, NX, Q1y, Q1x, zv = lattice_axes(c)
        mk = lambda nx: orc.Lattice(2, NX, N, nx, ny, orc.BC_WALLS,  # noqa: E731
                                    orc.tau_from_kn(N, ny, c["kn"], zv=zv & 2),
                                    c.get("u_wall_lo", 0.0), c.get("u_wall_hi", 0.0),
                                    c.get("g", 0.0), zv=zv, openmp=True)
        o = mk(1)
        X = o.equilibrium(np.ones((ny, 1)), np.zeros((ny, 1)), np.zeros((ny, 1)))
        t0 = time.perf_counter()
        o.run(X, 3)
        per_col = (time.perf_counter() - t0) / 3
        cols = int(max(1, min(c["nx"], budget / total_steps / max(per_col, 1e-9))))
        o = mk(cols)
        X = o.equilibrium(np.ones((ny, cols)), np.zeros((ny, cols)), np.zeros((ny, cols)))
        pops = Q1y * Q1x * ny * cols
        sample = f"{label}: strip of {cols} of {c['nx']} columns x {ny} rows, one instance, FP64"
    elif dims == 3:
        ny, nz = c["ny"], c["nz"]
        mk = lambda nx: orc.Lattice(3, N, N, nx, ny, orc.BC_WALLS,  # noqa: E731
                                    orc.tau_from_kn(N, ny, c["kn"]), c.get("u_wall_lo", 0.0),
                                    c.get("u_wall_hi", 0.0), c.get("g", 0.0), NZ=N, Lz=nz,
                                    openmp=True)
        o = mk(1)
        z1 = np.zeros((nz, ny, 1))
        t0 = time.perf_counter()
        o.run(o.equilibrium(z1 + 1, z1, z1, z1), 2)
        per_col = (time.perf_counter() - t0) / 2
        cols = int(max(1, min(c["nx"], budget / total_steps / max(per_col, 1e-9))))
        o = mk(cols)
        zc = np.zeros((nz, ny, cols))
        X = o.equilibrium(zc + 1, zc, zc, zc)
        pops = (2 * N + 1) ** 3 * ny * nz * cols
        sample = f"{label}: slab of {cols} of {c['nx']} x-columns ({ny} x {nz} each), one instance, FP64"
    else:
        o = orc.Lattice(1, N, 0, c["nx"], 1, orc.BC_BOUNCEBACK, orc.tau_from_kn(N, c["nx"], c["kn"]),
                        openmp=True)
        X = o.equilibrium(np.ones(c["nx"]), np.zeros(c["nx"]))
        pops = (2 * N + 1) * c["nx"]
        sample = f"{label}: full lattice, FP64"
    X, _ = o.run(X, args.warmup)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        X, _ = o.run(X, 1)
    dt = time.perf_counter() - t0
    value = pops * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args.workload, args, world),
            "reference": "FP64 CPU oracle (oracle/glbm_oracle.c)",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": _omp_threads(), "kind": "oracle",
                             "sample": sample + f", {_omp_threads()} threads (collision over rows)",
                             "host": _host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="couette",
                    choices=["couette", "couette_4096", "couette_aniso", "couette_zv",
                             "couette_zv_xy", "couette3d", "poiseuille", "sod", "batched",
                             "adjoint", "couette_slab"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--only", choices=["fp32", "fp64"], default=None,
                    help="time one precision's steps alone and print a reduced line (no "
                         "e2e, precision, batched or CPU baseline): for profiler captures")
    ap.add_argument("--tiles", default="autotune",
                    help="autotune (time every tile shape on the context first), default "
                         "(keep the defaults), or idx:<i> (FP32 candidate i of the level)")
    args = ap.parse_args()
    if args.tiles not in ("autotune", "default") and not (
            args.tiles.startswith("idx:") and args.tiles[4:].isdigit()):
        ap.error("--tiles takes autotune, default or idx:<i>")
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
