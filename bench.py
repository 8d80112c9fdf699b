"""Throughput benchmark of the IBLB hot path on GB300.

One "step" is one full IBLB time step of the 3D droplet workload
(D3Q19, 256 x 256 x 128 lattice, FP32 deviation storage, icosphere drop of
radius 40 with 10242 nodes / 20480 faces placed 42 lu above the wall,
theta_eq = 75 deg, tau = 0.8): nodal forces, spread, fused stream-collide,
interpolate + advect.  The population state (2 x 1.26 GB) is far larger than
L2, so no L2 flush is needed between steps.

Metric: MLUPS (million fluid-lattice-cell updates per second), whole job.
Also reported: the HBM-roofline fraction of the stream-collide kernel, an
end-to-end figure through the C-ABI with host buffers, and the FP64 CPU oracle
timed on a bounded sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Other modes (--mode), each printing one JSON line of its own:
  batch     256 uneven 2D drops: sequential FP32 vs batched FP32 / binary16
  serve     Poisson stream of 2D / 3D requests through the serving loop
  spread2d  2048x512 spreading sweep in FP64 / FP32 / binary16 storage, and
            the 4x-downscaled copy against the FP64 oracle
  spread3d  paper-scale 3D spreading (250x250x150 tau sweep, 300x300x250)
  shear     drop in shear flow at Re = 0.01, Ca = 0.05, R0 = 19 against Eq. 16
  profile   small cases for ncu captures (--case ib-cap | batch3d | batch2d | step3d)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_NAME = "d3q19_256x256x128_icosphere_R40_fp32dev"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e data-sheet figure, quoted beside the measured peak
TRAFFIC_FILES = {
    "fp32": os.path.join(ROOT, "profiles", "stream_collide_d3q19_256x256x128_fp32.txt"),
    "fp16": os.path.join(ROOT, "profiles", "stream_collide_d3q19_256x256x128_fp16.txt"),
}
CSRC = os.path.join(ROOT, "paper_2604_17463_gb300", "csrc")
SC_SOURCES = [os.path.join(CSRC, n) for n in ("lbm.cu", "lbm_pipe.cu", "lbm_core.cuh", "common.cuh")]


def hbm_peak():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def source_digest(paths):
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(storage, tuning=None):
    """Per-launch DRAM bytes of the stream-collide kernel from the committed ncu
    summary of the same storage form and kernel variant (the first field of
    the launch shape "variant,block_x,rows,ctas,warps"), valid only while the
    kernel source is unchanged since capture (None otherwise)."""
    try:
        vals = {}
        with open(TRAFFIC_FILES[storage]) as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("stream-collide sources sha256 prefix") != source_digest(SC_SOURCES):
            return None
        # the same kernel (variant); the block size does not change its traffic
        shape = vals.get("launch shape")
        if tuning is not None and shape is not None and shape.split(",")[0] != tuning.split(",")[0]:
            return None
        return float(vals["dram bytes per launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device: str = "cpu") -> float:
    """The maximum of a per-rank time over all ranks (replicas: the job ends
    when the slowest rank ends)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells_per_rank: int, steps: int, ms: float, world: int) -> float:
    """Whole-job throughput: every rank updates its own replica's cells."""
    return world * cells_per_rank * steps / (ms / 1e3) / 1e6


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def workload_config(wl, world):
    """The `config` object of both arms (the workload, not how it is run)."""
    return {"workload": WORKLOAD_NAME, "lattice": "D3Q19", "nx": wl.nx, "ny": wl.ny, "nz": wl.nz,
            "nodes": int(wl.nodes.shape[0]), "faces": int(wl.faces.shape[0]),
            "fluid_cells": wl.fluid_cells,
            "l2": "state (2 x 1.26 GB) larger than L2; no flush",
            "parallelism": f"replicas x{world}"}


def cpu_baseline_oracle(wl, steps, openmp=False):
    """FP64 CPU oracle on `steps` full time steps of the workload: one thread,
    or (openmp) its -fopenmp build on OMP_NUM_THREADS threads."""
    import oracle
    s = oracle.Sim(wl.lattice, wl.nx, wl.ny, wl.nz, tau=wl.tau, walls=wl.walls, wetting=wl.wetting,
                   sigma=wl.sigma, xi=wl.xi, theta_eq_deg=wl.theta_eq_deg, pi_n=wl.pi_n,
                   pi_m=wl.pi_m, openmp=openmp)
    s.set_interface(wl.nodes, wl.faces)
    t0 = time.perf_counter()
    rc = s.step(steps)
    dt = time.perf_counter() - t0
    s.close()
    if rc != 0:
        raise RuntimeError(f"oracle step failed: {rc}")
    return wl.fluid_cells * steps / dt / 1e6, dt


def run_reference(args, wl, budget_s=150.0):
    """The oracle timed on the host cores on the same workload and metric.
    A full 3D oracle step takes seconds, so at most as many steps as fit in
    `budget_s` are run (the metric is a rate; the sample is stated)."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    cores = host_cores()
    os.environ["OMP_NUM_THREADS"] = str(cores)
    import oracle
    s = oracle.Sim(wl.lattice, wl.nx, wl.ny, wl.nz, tau=wl.tau, walls=wl.walls, wetting=wl.wetting,
                   sigma=wl.sigma, xi=wl.xi, theta_eq_deg=wl.theta_eq_deg, pi_n=wl.pi_n,
                   pi_m=wl.pi_m, openmp=True)
    s.set_interface(wl.nodes, wl.faces)
    t0 = time.perf_counter()
    s.step(1)                                   # one untimed step sizes the sample
    per_step = time.perf_counter() - t0
    fit = max(1, int(budget_s / max(per_step, 1e-3)))
    warm = max(0, min(args.warmup, fit // 4) - 1)
    timed = max(1, min(args.steps, fit - warm))
    for _ in range(warm):
        s.step(1)
    t0 = time.perf_counter()
    for _ in range(timed):
        s.step(1)
    dt = time.perf_counter() - t0
    s.close()
    v = wl.fluid_cells * timed / dt / 1e6
    sample = (f"{timed} of {args.steps} requested full oracle time steps of the workload "
              f"(FP64; stream-collide rows on {cores} OpenMP threads, {dt:.1f} s)")
    line = {
        "impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": world,
        "steps": timed, "warmup": warm + 1, "ms_per_step": dt / timed * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(wl, world),
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, wl):
    import torch
    from paper_2604_17463_gb300 import iblb

    world, rank, local = dist_setup()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device (the CUDA library has no CPU path)")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    storage = {"fp32": iblb.FP32_DEV, "fp16": iblb.FP16_DEV, "fp64": iblb.FP64}[args.storage]
    sim = iblb.Simulation.from_workload(wl, storage=storage, stream=stream.cuda_stream)
    cells = sim.fluid_cells

    # ---- launch shape from the autotuner, then device-resident throughput (value)
    if args.tuning:
        v, bx, rows, ctas, ncw = (int(x) for x in args.tuning.split(","))
        sim.set_tuning(v, bx, 0, rows, ctas, ncw)
        tuned = sim.tuning()
        tuned["source"] = "fixed"
    else:
        tuned = sim.autotune(trials=10)
        tuned["source"] = "autotuner"
    # the library overlaps the IB kernels with the stream-collide of every
    # cell on 3D lattices of >= 2^20 cells (iblb_tuning.step_overlap = 0)
    overlapped = tuned["step_overlap"] == 1 or (
        tuned["step_overlap"] == 0 and wl.dim == 3 and wl.cells >= 1 << 20)
    sim.step(args.warmup)
    sim.sync()
    # The timed region is exactly `steps` steps, bracketed by a barrier and a
    # synchronisation; it is repeated until at least one second of device
    # time has passed (so that the clock sampler sees the GPU under load) and
    # the median repetition is reported.
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps, launches = [], 0
    with ClockSampler(local) as clk:
        while True:
            n0 = iblb.iblb_kernel_launch_count()
            barrier()
            torch.cuda.synchronize()
            ev0.record(stream)
            sim.step(args.steps)
            ev1.record(stream)
            ev1.synchronize()
            torch.cuda.synchronize()
            barrier()
            launches = iblb.iblb_kernel_launch_count() - n0
            reps.append(max_over_ranks(ev0.elapsed_time(ev1), world, device="cuda"))
            if (sum(reps) >= 1000.0 and len(reps) >= 3) or len(reps) >= 2000:
                break
    sim.sync()
    ms = statistics.median(reps)
    ms_per_step = ms / args.steps
    value = whole_job_mlups(cells, args.steps, ms, world)

    # ---- per-kernel device times (CUDA events around each launch)
    prof_steps = max(5, min(args.steps, 200))
    kms = sim.step_profiled(prof_steps)
    sc_ms = kms[iblb.K_STREAM_COLLIDE] / prof_steps
    bytes_per_launch = sim.stream_bytes_per_step
    achieved = bytes_per_launch / (sc_ms / 1e3) / 1e9
    peak, peak_kind = hbm_peak()
    kernel_share = {iblb.KERNEL_NAMES[k]: kms[k] / kms.sum() for k in range(iblb.K_COUNT)}
    sim.close()

    # ---- end to end through the C-ABI with pinned host buffers
    xyz_host = torch.from_numpy(np.ascontiguousarray(wl.nodes)).pin_memory().numpy()
    ncell = wl.cells
    rho_out = torch.empty(ncell, dtype=torch.float64).pin_memory().numpy()
    u_out = torch.empty(3 * ncell, dtype=torch.float64).pin_memory().numpy()
    xyz_out = torch.empty(wl.nodes.size, dtype=torch.float64).pin_memory().numpy()
    tri = np.ascontiguousarray(wl.faces, dtype=np.int32)
    sim2 = iblb.Simulation(wl.lattice, wl.nx, wl.ny, wl.nz, stream=stream.cuda_stream,
                           tau=wl.tau, walls=wl.walls, wetting=wl.wetting, sigma=wl.sigma,
                           xi=wl.xi, theta_eq_deg=wl.theta_eq_deg, pi_n=wl.pi_n, pi_m=wl.pi_m,
                           storage=storage)
    sim2.set_interface(xyz_host, tri)
    sim2.set_tuning(tuned["variant"], tuned["block_x"], 0, tuned["rows_per_tile"],
                    tuned["ctas_per_sm"], tuned["consumer_warps"])
    sim2.step(args.warmup)
    sim2.sync()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iblb.iblb_set_interface(sim2.h, xyz_host, tri)
    iblb.iblb_step(sim2.h, args.steps)
    iblb.iblb_read_fields(sim2.h, rho_out, u_out, xyz_out)
    e2e_s = time.perf_counter() - t0
    barrier()
    sim2.close()
    e2e_value = world * cells * args.steps / e2e_s / 1e6
    h2d = (xyz_host.nbytes + tri.nbytes) / args.steps
    d2h = (rho_out.nbytes + u_out.nbytes + xyz_out.nbytes) / args.steps

    batch = None
    if world == 1 and not args.no_batch:
        batch = batch_object(args)
    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        os.environ["OMP_NUM_THREADS"] = str(cores)
        cpu_steps = 3
        cv, cdt = cpu_baseline_oracle(wl, cpu_steps, openmp=True)
        c1v, c1dt = cpu_baseline_oracle(wl, 2)
        from paper_2604_17463_gb300 import workloads as W
        c1, _ = cpu_baseline_oracle(W.drop_2d_128x64(), 200)
        c2d, _ = cpu_baseline_oracle(W.spreading_2d_2048x512(downscale=4), 50)
        cpu = {"value": cv, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{cpu_steps} full time steps of the same workload in the FP64 oracle "
                         f"(stream-collide rows on {cores} OpenMP threads, {cdt:.1f} s)",
               "single_thread": {"value": c1v, "unit": "MLUPS", "cores": 1,
                                 "sample": f"2 full time steps, one thread, {c1dt:.1f} s"},
               "other_workloads_mlups": {"d2q9_128x64 drop (200 steps, 1 thread)": c1,
                                         "d2q9_512x128 spreading, 2048x512 downscaled 4x (50 steps, 1 thread)": c2d}}
    clocks = clk.summary()
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f32 (binary16 storage)", "fp64": "f64"}[args.storage],
        "data": "synthetic",
        "config": workload_config(wl, world),
        "storage": args.storage,
        "stream_collide_tuning": tuned,
        "overlapped_step": overlapped,
        "timing": {"repeats": len(reps), "ms_per_repeat_min": min(reps),
                   "ms_per_repeat_max": max(reps), "statistic": "median of the repeats"},
        "roofline": {"bound": "hbm",
                     "kernel": "stream_collide (bulk pass)" if overlapped else "stream_collide",
                     "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": ncu_traffic(args.storage, ",".join(
                         str(tuned[k]) for k in ("variant", "block_x", "rows_per_tile",
                                                 "ctas_per_sm", "consumer_warps"))),
                     "bytes_per_launch": bytes_per_launch, "launch_ms": sc_ms,
                     "stream_collide_mlups": cells / (sc_ms * 1e-3) / 1e6,
                     "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "kernel_share": kernel_share},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cpu_baseline": cpu,
        "batch": batch,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batch_object(args):
    """The batched engine on the 256-drop workload (widths 64-1024
    log-uniform, height w/4) at its stated step counts U[5000, 50000]:
    - the batched stream-collide kernel against the HBM bound with every
      slot active (algorithmic bytes of all slots / CUDA-event launch time),
      FP32 and binary16 storage;
    - whole-set runs, batched FP32 and batched binary16: sims/hour;
    - the one-simulation-at-a-time FP32 path on a seeded sample of the set
      (sims/hour of that sample), and the largest contact-angle difference of
      each batched form to those sequential runs."""
    import torch
    from paper_2604_17463_gb300 import iblb, serve
    from paper_2604_17463_gb300 import workloads as W
    wls = W.batch_2d_drops()
    stream = torch.cuda.current_stream().cuda_stream
    peak, kind = hbm_peak()
    budget = 24 << 30
    out = {"workload": f"{len(wls)} D2Q9 drops, widths 64-1024 log-uniform, height w/4, "
                       "steps U[5000, 50000]", "kernel": {}}
    cells = sum(w.fluid_cells for w in wls)
    for name, st in (("fp32", iblb.FP32_DEV), ("fp16", iblb.FP16_DEV)):
        b = iblb.Batch(iblb.D2Q9, st, budget, max_slots=len(wls) + 8, stream=stream)
        for wl in wls:
            if b.admit_workload(wl) is None:
                raise RuntimeError("the batch budget does not hold the 256-drop set")
        b.run_profiled(3)
        steps = 20
        _, kms, nbytes = b.run_profiled(steps)
        b.close()
        sc_ms = kms[iblb.K_STREAM_COLLIDE] / steps
        achieved = nbytes / steps / (sc_ms * 1e-3) / 1e9
        out["kernel"][name] = {"bound": "hbm", "achieved": achieved, "peak": peak,
                               "peak_kind": kind, "unit": "GB/s", "frac": achieved / peak,
                               "launch_ms": sc_ms, "bytes_per_launch": nbytes / steps,
                               "glups": cells / (sc_ms * 1e-3) / 1e9,
                               "phase_ms": {iblb.KERNEL_NAMES[k]: kms[k] / steps
                                            for k in range(iblb.K_COUNT)}}
    rng = np.random.default_rng(20260417 + 40)
    idx = sorted(int(i) for i in rng.choice(len(wls), size=min(args.batch_seq_sample, len(wls)),
                                            replace=False))
    seq = serve.run_sequential([wls[i] for i in idx], iblb.FP32_DEV, stream=stream)
    b32 = serve.run_batched(wls, iblb.FP32_DEV, budget, stream=stream)
    b16 = serve.run_batched(wls, iblb.FP16_DEV, budget, stream=stream)

    def dtheta(run):
        d = [abs(run["obs"][i]["theta_deg"] - o["theta_deg"]) for i, o in zip(idx, seq["obs"])
             if np.isfinite(o["theta_deg"]) and np.isfinite(run["obs"][i]["theta_deg"])]
        return (max(d) if d else None), len(d)

    cell_steps = sum(w.fluid_cells * w.steps for w in wls)
    seq_cell_steps = sum(wls[i].fluid_cells * wls[i].steps for i in idx)
    out["sequential_fp32"] = {"sims_per_hour": len(idx) / seq["wall_s"] * 3600,
                              "wall_s": seq["wall_s"], "mlups": seq_cell_steps / seq["wall_s"] / 1e6,
                              "sample": f"{len(idx)} of the {len(wls)} drops (seeded), one at a time"}
    for name, run in (("batched_fp32", b32), ("batched_fp16", b16)):
        d, n = dtheta(run)
        out[name] = {"sims_per_hour": len(wls) / run["wall_s"] * 3600, "wall_s": run["wall_s"],
                     "mlups": cell_steps / run["wall_s"] / 1e6,
                     "max_dtheta_deg_vs_sequential_fp32": d, "compared": n}
    out["speedup_fp16_batch_vs_sequential_fp32"] = (
        out["batched_fp16"]["sims_per_hour"] / out["sequential_fp32"]["sims_per_hour"])
    return out


def run_batch_mode(args):
    """Batched engine on the 256-drop workload (widths 64-1024, step counts
    scaled by 1/step_div): sequential single-engine FP32 vs batched FP32 and
    batched binary16 storage; sims/hour and the contact-angle difference of
    the reduced-precision batch against the sequential FP32 runs."""
    import torch
    from paper_2604_17463_gb300 import iblb, serve
    from paper_2604_17463_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    wls = W.batch_2d_drops(count=args.count, steps_lo=5000 // args.step_div, steps_hi=50000 // args.step_div)
    stream = torch.cuda.current_stream().cuda_stream
    n0 = iblb.iblb_kernel_launch_count()
    seq = serve.run_sequential(wls, iblb.FP32_DEV, stream=stream)
    b32 = serve.run_batched(wls, iblb.FP32_DEV, 16 << 30, stream=stream)
    b16 = serve.run_batched(wls, iblb.FP16_DEV, 16 << 30, stream=stream)
    launches = iblb.iblb_kernel_launch_count() - n0

    def dtheta(a, b):
        d = [abs(x["theta_deg"] - y["theta_deg"]) for x, y in zip(a["obs"], b["obs"])
             if np.isfinite(x["theta_deg"]) and np.isfinite(y["theta_deg"])]
        return max(d) if d else None, len(d)

    cells_steps = sum(w.fluid_cells * w.steps for w in wls)
    d16, n16 = dtheta(b16, seq)
    d32, n32 = dtheta(b32, seq)
    line = {
        "metric": "sims_per_hour", "value": len(wls) / b16["wall_s"] * 3600, "unit": "sims/h",
        "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "f32 (binary16 storage)",
        "config": {"workload": f"{len(wls)} D2Q9 drops, widths 64-1024 log-uniform, height w/4, "
                               f"steps U[{5000 // args.step_div}, {50000 // args.step_div}]",
                   "mode": "batch"},
        "sequential_fp32": {"sims_per_hour": len(wls) / seq["wall_s"] * 3600, "wall_s": seq["wall_s"],
                            "mlups": cells_steps / seq["wall_s"] / 1e6},
        "batched_fp32": {"sims_per_hour": len(wls) / b32["wall_s"] * 3600, "wall_s": b32["wall_s"],
                         "mlups": cells_steps / b32["wall_s"] / 1e6, "max_dtheta_deg_vs_seq": d32,
                         "compared": n32},
        "batched_fp16": {"sims_per_hour": len(wls) / b16["wall_s"] * 3600, "wall_s": b16["wall_s"],
                         "mlups": cells_steps / b16["wall_s"] / 1e6, "max_dtheta_deg_vs_seq": d16,
                         "compared": n16},
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    return 0


def _oracle_request(job):
    """FP64 oracle run of one 2D serving request (in a spawned worker):
    its contact angle and height after its step count."""
    nx, ny, tau, sigma, xi, theta, pi_n, pi_m, steps, nodes = job
    import oracle
    o = oracle.Sim(9, nx, ny, tau=tau, sigma=sigma, xi=xi, theta_eq_deg=theta, pi_n=pi_n,
                   pi_m=pi_m)
    o.set_interface(nodes)
    rc = o.step(steps)
    ob = o.observables()
    o.close()
    return rc, ob["theta_deg"], ob["height"]


def run_serve_mode(args):
    """Serving loop on a Poisson stream of wetting requests (80 % 2D as the
    batched workload, 20 % D3Q19 between 64^3 and 192x192x96; step counts
    U[5000, 50000] / step_div); the contact angle and height of a seeded
    sample of the 2D requests (args.oracle_frac of them) against the FP64
    oracle, run on the host cores in spawned workers while the GPU serves."""
    import multiprocessing as mp

    import torch
    from paper_2604_17463_gb300 import iblb, serve
    from paper_2604_17463_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    reqs = W.serve_requests(count=args.count, rate_per_s=args.rate, steps_lo=5000 // args.step_div,
                     steps_hi=50000 // args.step_div)
    storage = {"fp32": iblb.FP32_DEV, "fp16": iblb.FP16_DEV, "fp64": iblb.FP64}[args.serve_storage]
    # seeded sample of the 2D requests for the oracle check (among those the
    # single-threaded oracle runs in a bounded time)
    two_d = [i for i, r in enumerate(reqs) if r.work.lattice == 9 and
             r.work.fluid_cells * r.work.steps <= args.oracle_max_updates]
    k = max(1, int(round(args.oracle_frac * len(reqs))))
    rng = np.random.default_rng(20260417 + 55)
    sample = sorted(int(i) for i in rng.choice(two_d, size=min(k, len(two_d)), replace=False))
    jobs = [(w.nx, w.ny, w.tau, w.sigma, w.xi, w.theta_eq_deg, w.pi_n, w.pi_m, w.steps, w.nodes)
            for w in (reqs[i].work for i in sample)]
    cores = host_cores()
    pool = mp.get_context("spawn").Pool(processes=max(1, min(len(jobs), cores - 1)))
    pending = pool.map_async(_oracle_request, jobs, chunksize=1)
    n0 = iblb.iblb_kernel_launch_count()
    out = serve.serve(reqs, storage, budget_2d=24 << 30, budget_3d=96 << 30, chunk=args.chunk)
    launches = iblb.iblb_kernel_launch_count() - n0
    t_wait = time.perf_counter()
    oracle_out = pending.get()
    oracle_extra_s = time.perf_counter() - t_wait
    pool.close()
    pool.join()
    errs, herrs = [], []
    for i, (rc, th, h) in zip(sample, oracle_out):
        got = out["results"][i]
        if rc != 0:
            continue
        herrs.append(abs(h - got["height"]) / h)
        # the angle is meaningful once the drop sits on its film (below 175 deg)
        if np.isfinite(th) and th < 175.0:
            errs.append(abs(th - got["theta_deg"]))
    line = {
        "metric": "sims_per_hour", "value": out["sims_per_hour"], "unit": "sims/h", "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic",
        "dtype": {"fp32": "f32", "fp16": "f32 (binary16 storage)", "fp64": "f64"}[args.serve_storage],
        "config": {"workload": f"{len(reqs)} Poisson requests at {args.rate}/s, 80% D2Q9 "
                               f"(w 64-1024), 20% D3Q19 (64^3-192x192x96), steps "
                               f"U[{5000 // args.step_div}, {50000 // args.step_div}]",
                   "mode": "serve", "chunk_steps": args.chunk},
        "p50_s": out["p50_s"], "p99_s": out["p99_s"], "wall_s": out["wall_s"],
        "completed": out["completed"], "mlups": out["mlups"], "max_queue": out["max_queue"],
        "oracle_check": {"max_dtheta_deg": max(errs) if errs else None, "theta_compared": len(errs),
                         "max_rel_dheight": max(herrs) if herrs else None,
                         "requests": len(sample), "sample": f"seeded {len(sample)} of the "
                         f"{len(two_d)} 2D requests with at most {args.oracle_max_updates:.0e} "
                         f"cell updates ({args.oracle_frac:.0%} of all requests)",
                         "oracle_cores": pool._processes if hasattr(pool, "_processes") else None,
                         "oracle_wait_after_serving_s": oracle_extra_s},
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    return 0


def _oracle_spread_trajectory(job):
    """Oracle trajectory of one downscaled spreading case (runs in a spawned
    worker process): observables at each checkpoint."""
    theta, tau, steps, checkpoints = job
    import oracle
    from paper_2604_17463_gb300 import workloads as W
    wl = W.spreading_2d_2048x512(theta_eq_deg=theta, tau=tau, downscale=4)
    o = oracle.Sim(9, wl.nx, wl.ny, tau=wl.tau, sigma=wl.sigma, xi=wl.xi,
                   theta_eq_deg=wl.theta_eq_deg, pi_n=wl.pi_n, pi_m=wl.pi_m)
    o.set_interface(wl.nodes)
    out = []
    for _ in range(checkpoints):
        o.step(steps // checkpoints)
        out.append(o.observables())
    o.close()
    return out


def run_spread2d_mode(args):
    """The 2D spreading sweep (2048x512 D2Q9, R = 200, 2000 nodes, initial
    angle 150 deg; theta_eq in {30, 60, 90, 120}, tau in {0.6, 1.0}; 200k
    steps / step_div): FP64, FP32 and binary16 storage on the GPU, contact
    angle, contact-line radius and film against the FP64 GPU run along the
    whole run; and the 4x-downscaled copy (512x128, 200k/16 steps / step_div,
    the same number of viscous times) in FP32 / binary16 against the FP64
    oracle, whose runs go to spawned worker processes started before the
    first GPU call."""
    import multiprocessing as mp
    thetas, taus = (30.0, 60.0, 90.0, 120.0), (0.6, 1.0)
    combos = [(t, tau) for t in thetas for tau in taus]
    cps = 20
    steps_full = 200000 // args.step_div
    steps_ds = 200000 // 16 // args.step_div
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(min(len(combos), os.cpu_count() or 1))
    t_or = time.perf_counter()
    pending = pool.map_async(_oracle_spread_trajectory,
                             [(t, tau, steps_ds, cps) for t, tau in combos])
    import torch
    from paper_2604_17463_gb300 import iblb
    from paper_2604_17463_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    names = {iblb.FP64: "fp64", iblb.FP32_DEV: "fp32", iblb.FP16_DEV: "fp16"}
    n0 = iblb.iblb_kernel_launch_count()

    def traj(wl, storage, steps):
        g = iblb.Simulation.from_workload(wl, storage=storage, stream=stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out = []
        e0.record(stream)
        for _ in range(cps):
            g.step(steps // cps)
            out.append(g.observables())
        e1.record(stream)
        torch.cuda.synchronize()
        g.close()
        return out, e0.elapsed_time(e1) * 1e-3

    def compare(got, ref, xi):
        dth = [abs(a["theta_deg"] - b["theta_deg"]) for a, b in zip(got, ref)
               if np.isfinite(a["theta_deg"]) and np.isfinite(b["theta_deg"])]
        drc = [abs(a["r_cl"] - b["r_cl"]) / max(b["r_cl"], 1.0) for a, b in zip(got, ref)]
        dfilm = [abs(a["film"] - b["film"]) / xi for a, b in zip(got, ref)
                 if np.isfinite(a["film"]) and np.isfinite(b["film"])]
        return {"max_dtheta_deg": max(dth) if dth else None,
                "max_rel_dr_cl": max(drc), "max_dfilm_over_xi": max(dfilm) if dfilm else None}

    full, ds = [], []
    dev_s = {n: 0.0 for n in names.values()}
    for theta, tau in combos:
        wl = W.spreading_2d_2048x512(theta_eq_deg=theta, tau=tau)
        runs = {}
        for st in (iblb.FP64, iblb.FP32_DEV, iblb.FP16_DEV):
            runs[st], sec = traj(wl, st, steps_full)
            dev_s[names[st]] += sec
        ref = runs[iblb.FP64]
        # a second FP64 run: the spread's atomics add in a different order, so
        # this is the run-to-run spread of the FP64 path itself
        rep, _ = traj(wl, iblb.FP64, steps_full)
        full.append({"theta_eq": theta, "tau": tau,
                     "fp64_repeat_vs_fp64": compare(rep, ref, wl.xi),
                     "fp32_vs_fp64": compare(runs[iblb.FP32_DEV], ref, wl.xi),
                     "fp16_vs_fp64": compare(runs[iblb.FP16_DEV], ref, wl.xi),
                     "final": {n: {k: runs[st][-1][k] for k in ("theta_deg", "r_cl", "film")}
                               for st, n in names.items()},
                     "theta_t_fp16": [round(o["theta_deg"], 3) for o in runs[iblb.FP16_DEV]]})
        wd = W.spreading_2d_2048x512(theta_eq_deg=theta, tau=tau, downscale=4)
        ds.append({"theta_eq": theta, "tau": tau, "wl": wd,
                   "gpu": {st: traj(wd, st, steps_ds)[0] for st in (iblb.FP32_DEV, iblb.FP16_DEV)}})
    launches = iblb.iblb_kernel_launch_count() - n0
    oracle_runs = pending.get()
    pool.close()
    t_or = time.perf_counter() - t_or
    for d, orc in zip(ds, oracle_runs):
        d["fp32_vs_oracle"] = compare(d["gpu"][iblb.FP32_DEV], orc, d["wl"].xi)
        d["fp16_vs_oracle"] = compare(d["gpu"][iblb.FP16_DEV], orc, d["wl"].xi)
        d["oracle_final_theta"] = orc[-1]["theta_deg"]
        del d["gpu"], d["wl"]
    cells = 2048 * 510
    worst16 = max(f["fp16_vs_fp64"]["max_dtheta_deg"] or 0.0 for f in full)
    line = {
        "metric": "max_dtheta_deg_fp16_vs_fp64", "value": worst16, "unit": "deg", "n_gpus": 1,
        "higher_is_better": False, "data": "synthetic", "dtype": "f32 (fp64 / fp32 / binary16 storage)",
        "config": {"workload": f"D2Q9 2048x512 spreading, R = 200, 2000 nodes, 150 deg start, "
                               f"theta_eq {list(thetas)}, tau {list(taus)}, {steps_full} steps; "
                               f"oracle on the 512x128 copy, {steps_ds} steps",
                   "mode": "spread2d", "checkpoints": cps},
        "mlups": {n: len(combos) * cells * steps_full / dev_s[n] / 1e6 for n in names.values()},
        "full_size": full, "downscaled_vs_oracle": ds, "oracle_wall_s": t_or,
        "oracle_processes": min(len(combos), os.cpu_count() or 1),
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_spread3d_mode(args):
    """Paper-scale 3D spreading (Sec. 3: 250x250x150, a hemisphere of R0 = 50
    on its film spreading to 60 deg, about 120 000 triangles, tau in {0.56,
    0.59, 0.732, 1.1}; Sec. 4: 300x300x250, a sphere at the film distance
    spreading to 45 deg at tau = 0.56), FP32 storage: h(t)/R0 over
    --spread3d-t-mu capillary times, throughput per run, and the per-kernel
    split of one step on the first lattice."""
    import torch
    from paper_2604_17463_gb300 import iblb
    from paper_2604_17463_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    storage = {"fp32": iblb.FP32_DEV, "fp16": iblb.FP16_DEV, "fp64": iblb.FP64}[args.storage]
    taus = [float(t) for t in args.spread3d_taus.split(",") if t]
    cases = [W.spread3d_cap(t, t_mu_count=args.spread3d_t_mu) for t in taus]
    if args.spread3d_sphere:
        cases.append(W.spread3d_sphere(t_mu_count=args.spread3d_t_mu))
    n0 = iblb.iblb_kernel_launch_count()
    runs = []
    gp = iblb.Simulation.from_workload(cases[0].work, storage=storage, stream=stream.cuda_stream)
    ms = gp.step_profiled(50)
    gp.close()
    tot = float(ms.sum())
    split = {k: float(v) / tot for k, v in zip(iblb.KERNEL_NAMES, ms)}
    split["ms_per_step"] = tot / 50
    for case in cases:
        wl = case.work
        g = iblb.Simulation.from_workload(wl, storage=storage, stream=stream.cuda_stream)
        samples = 100
        per = max(1, wl.steps // samples)
        hist = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(samples):
            g.step(per)
            o = g.observables()
            hist.append([round((k + 1) * per / case.t_mu, 3), round(o["height"] / case.R0, 5),
                         round(o["theta_deg"], 3)])
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        o = g.observables()
        g.close()
        hs = [h[1] for h in hist]
        runs.append({"workload": wl.name, "tau": wl.tau, "Re": case.Re, "t_mu_steps": case.t_mu,
                     "steps": per * samples, "nodes": len(wl.nodes), "faces": len(wl.faces),
                     "mlups": wl.fluid_cells * per * samples / sec / 1e6, "device_s": sec,
                     "h_over_R0_final": hs[-1], "h_over_R0_min": min(hs),
                     "theta_final_deg": o["theta_deg"],
                     "h_over_R0_t": hist})
    launches = iblb.iblb_kernel_launch_count() - n0
    cells = sum(c.work.fluid_cells * r["steps"] for c, r in zip(cases, runs))
    secs = sum(r["device_s"] for r in runs)
    line = {
        "metric": "mlups", "value": cells / secs / 1e6, "unit": "MLUPS", "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic",
        "dtype": {"fp32": "f32", "fp16": "f32 (binary16 storage)", "fp64": "f64"}[args.storage],
        "config": {"workload": "paper-scale 3D spreading: 250x250x150 hemisphere R0 = 50 -> 60 deg, "
                               f"tau {taus}" + (", 300x300x250 sphere -> 45 deg, tau 0.56"
                                                if args.spread3d_sphere else "")
                               + f", ~120k triangles, {args.spread3d_t_mu:g} t_mu each",
                   "mode": "spread3d"},
        "step_split_first_lattice": split, "runs": runs, "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_profile_mode(args):
    """Small cases of the 3D kernels for profiler captures (ncu): a few
    profiled steps (no graphs), one JSON line of per-phase device times.
      ib-cap   the paper-scale cap mesh (59 292 nodes, 118 580 faces) moved
               into a 128 x 128 x 64 lattice, FP32 storage, per-node IB
               kernels (--ib-grouped 1: grouped)
      batch3d  the first 8 D3Q19 requests of the serving mix in one batch
               of storage --storage (default FP32); the profiled steps run
               inside the NVTX range "run"
      batch2d  the 256 D2Q9 drops of the batched workload in one batch of
               storage --storage, likewise inside the NVTX range "run"
      step3d   a 3D drop on a 192 x 192 x 96 lattice (R = 30, 10 242 nodes;
               0.54 GB of FP32 populations, above L2), storage --storage,
               the overlapped step's kernels (bulk pass with the launch
               shape of --tuning, default the x-pair kernel for FP32 and
               the row-pair kernel for binary16, then the band pass)
    """
    import dataclasses
    import torch
    from paper_2604_17463_gb300 import iblb
    from paper_2604_17463_gb300 import workloads as W
    torch.cuda.set_device(0)
    out = {"mode": "profile", "case": args.case}
    if args.case == "ib-cap":
        wl = W.spread3d_cap(0.59).work
        wl = dataclasses.replace(wl, nx=128, ny=128, nz=64,
                                 nodes=wl.nodes - [125.0 - 64.0, 125.0 - 64.0, 0.0])
        sim = iblb.Simulation.from_workload(wl, storage=iblb.FP32_DEV)
        sim.set_tuning(0, 64, ib_grouped=args.ib_grouped, step_overlap=2)
        steps = 6
        kms = sim.step_profiled(steps) / steps
        out.update(nodes=int(wl.nodes.shape[0]), faces=int(wl.faces.shape[0]),
                   lattice=[wl.nx, wl.ny, wl.nz])
        sim.close()
    elif args.case == "step3d":
        nodes, faces = W.icosphere(5, 30.0, (96.0 + 0.31, 96.0 - 0.22, W.WALL_PLANE + 32.0))
        wl = W.Workload("step3d_192x192x96", 19, 192, 192, 96, 0.8, 1e-3, 1.0, 75.0, 9, 3, 100,
                        nodes, faces)
        storage = {"fp32": iblb.FP32_DEV, "fp16": iblb.FP16_DEV, "fp64": iblb.FP64}[args.storage]
        sim = iblb.Simulation.from_workload(wl, storage=storage)
        default = "3,128,2,2,8" if args.storage == "fp16" else "2,128,2,2,8"
        v, bx, rows, ctas, ncw = (int(x) for x in (args.tuning or default).split(","))
        sim.set_tuning(v, bx, 0, rows, ctas, ncw, step_overlap=1)
        steps = 6
        kms = sim.step_profiled(steps) / steps
        out.update(nodes=int(nodes.shape[0]), lattice=[wl.nx, wl.ny, wl.nz],
                   tuning=sim.tuning(), fluid_cells=int(sim.fluid_cells))
        sim.close()
    else:
        if args.case == "batch2d":
            wls, lat = W.batch_2d_drops(), iblb.D2Q9
        else:
            reqs = W.serve_requests(count=2000, rate_per_s=1.0)
            wls, lat = [r.work for r in reqs if r.work.lattice == 19][:8], iblb.D3Q19
        storage = {"fp32": iblb.FP32_DEV, "fp16": iblb.FP16_DEV, "fp64": iblb.FP64}[args.storage]
        b = iblb.Batch(lat, storage, 8 << 30, max_slots=len(wls) + 8)
        for w in wls:
            if b.admit_workload(w, n_steps=100000) is None:
                raise RuntimeError("batch3d: a request did not fit")
        steps = 4
        torch.cuda.nvtx.range_push("run")
        _, kms, _ = b.run_profiled(steps)
        b.sync()
        torch.cuda.nvtx.range_pop()
        kms = kms / steps
        out.update(slots=len(wls), storage=args.storage,
                   fluid_cells=int(sum(w.fluid_cells for w in wls)))
        b.close()
    out["phase_ms"] = {iblb.KERNEL_NAMES[k]: float(kms[k]) for k in range(iblb.K_COUNT)}
    print(json.dumps(out))
    return 0


def run_kernel2d_mode(args):
    """Stream-collide alone on a plain D2Q9 lattice (--nx x --ny, walls, no
    interface), the launch shape from --tuning or the autotuner: the 2D
    roofline point.  Device time of the kernel from CUDA events."""
    import torch
    from paper_2604_17463_gb300 import iblb
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    storage = {"fp32": iblb.FP32_DEV, "fp16": iblb.FP16_DEV, "fp64": iblb.FP64}[args.storage]
    stream = torch.cuda.current_stream()
    g = iblb.Simulation(9, args.nx, args.ny, tau=0.8, wetting=False, sigma=0.0,
                        body_force=(1e-6, 0.0, 0.0), storage=storage, stream=stream.cuda_stream)
    if args.tuning:
        v, bx, rows, ctas, ncw = (int(x) for x in args.tuning.split(","))
        g.set_tuning(v, bx, 0, rows, ctas, ncw)
        tuned = g.tuning()
    else:
        tuned = g.autotune(trials=5)
    g.step(args.warmup)
    n0 = iblb.iblb_kernel_launch_count()
    ms = g.step_profiled(args.steps)
    launches = iblb.iblb_kernel_launch_count() - n0
    sc_ms = float(ms[iblb.K_STREAM_COLLIDE]) / args.steps
    cells = g.fluid_cells
    bytes_per_launch = g.stream_bytes_per_step
    g.close()
    peak, peak_kind = hbm_peak()
    achieved = bytes_per_launch / (sc_ms * 1e-3) / 1e9
    line = {
        "metric": "mlups", "value": cells / (sc_ms * 1e-3) / 1e6, "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "data": "synthetic", "dtype": {"fp32": "f32", "fp16": "f32 (binary16 storage)",
                                       "fp64": "f64"}[args.storage],
        "config": {"workload": f"D2Q9 {args.nx}x{args.ny} stream-collide alone (walls, body "
                               f"force, no interface)", "mode": "kernel2d",
                   "stream_collide_tuning": tuned},
        "roofline": {"bound": "hbm",
                     "kernel": "stream_collide (bulk pass)" if overlapped else "stream_collide",
                     "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "bytes_per_launch": bytes_per_launch, "launch_ms": sc_ms},
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_shear_mode(args):
    """Drop in shear at the paper's parameters (Sec. 4: Re = 0.01, Ca = 0.05,
    R0 = 19, tau = 1, lambda from --shear-lam): moving-wall bounce-back, the
    fully developed linear profile as initial state, D (Eq. 15) sampled 24
    times, the last sample against Eq. 16.  Throughput is fluid-cell updates
    per second over the whole run (every step, every sample)."""
    import torch
    from paper_2604_17463_gb300 import iblb
    from paper_2604_17463_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    tau = 1.0
    tau_out = 0.5 + (tau - 0.5) / args.shear_lam
    case = W.shear_drop(tau=tau, tau_out=tau_out, t_mu_count=args.shear_t_mu)
    wl = case.work
    storage = {"fp32": iblb.FP32_DEV, "fp16": iblb.FP16_DEV, "fp64": iblb.FP64}[args.storage]
    stream = torch.cuda.current_stream()
    g = iblb.Simulation.from_workload(wl, storage=storage, stream=stream.cuda_stream,
                                      tau_out=case.tau_out, wall_u_lo=case.wall_u_lo,
                                      wall_u_hi=case.wall_u_hi)
    g.set_equilibrium(case.initial_velocity())
    samples = 24
    per = wl.steps // samples
    n0 = iblb.iblb_kernel_launch_count()
    hist = []
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(stream)
    for k in range(samples):
        g.step(per)
        d = g.deformation()
        hist.append([round((k + 1) * per / case.t_mu, 3), d["D"], d["angle_deg"]])
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = ev0.elapsed_time(ev1)
    launches = iblb.iblb_kernel_launch_count() - n0
    g.close()
    steps = per * samples
    D_end, D_inf = hist[-1][1], case.d_inf()
    line = {
        "metric": "mlups", "value": wl.fluid_cells * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
        "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
        "dtype": {"fp32": "f32", "fp16": "f32 (binary16 storage)", "fp64": "f64"}[args.storage],
        "config": {"workload": f"drop in shear, D3Q19 {wl.nx}x{wl.ny}x{wl.nz}, R0 = {case.R0:g}, "
                               f"{len(wl.nodes)} nodes, Re = {case.Re:g}, Ca = {case.Ca:g}, "
                               f"lambda = {case.lam:g}, {steps} steps ({args.shear_t_mu:g} t_mu)",
                   "mode": "shear"},
        "D_end": D_end, "D_inf_eq13": D_inf, "rel_distance": abs(D_end - D_inf) / D_inf,
        "inclination_deg": hist[-1][2], "device_s": ms * 1e-3, "wall_s": wall,
        "history_t_over_t_mu_D_angle": hist, "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="leave out the batched-engine object of the default line")
    ap.add_argument("--batch-seq-sample", type=int, default=48,
                    help="drops of the 256-drop set run one at a time for the sequential FP32 "
                         "baseline of the batch object")
    ap.add_argument("--mode", default="step", choices=["step", "batch", "serve", "shear", "spread2d", "spread3d",
                             "kernel2d", "profile"],
                    help="step: the 3D workload (default); batch / serve: the batched "
                         "and served engines; spread2d / spread3d: the 2D precision sweep "
                         "and the paper-scale 3D spreading runs; shear: the drop in shear")
    ap.add_argument("--count", type=int, default=256, help="batch / serve: simulations")
    ap.add_argument("--step-div", type=int, default=10,
                    help="batch / serve / spread2d: divide the step counts by this")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: arrivals per second")
    ap.add_argument("--chunk", type=int, default=500, help="serve: steps per scheduling round")
    ap.add_argument("--oracle-max-updates", type=float, default=3e9,
                    help="serve: the oracle sample is drawn among the 2D requests with at most "
                         "this many cell updates")
    ap.add_argument("--oracle-frac", type=float, default=0.02,
                    help="serve: fraction of the requests (drawn among the 2D ones) checked "
                         "against the FP64 oracle")
    ap.add_argument("--serve-storage", default="fp16", choices=["fp32", "fp16", "fp64"])
    ap.add_argument("--shear-lam", type=float, default=1.0, help="shear: viscosity ratio")
    ap.add_argument("--nx", type=int, default=4096, help="kernel2d: lattice width")
    ap.add_argument("--ny", type=int, default=4096, help="kernel2d: lattice height")
    ap.add_argument("--spread3d-taus", default="0.56,0.59,0.732,1.1",
                    help="spread3d: relaxation times of the 250x250x150 runs")
    ap.add_argument("--spread3d-sphere", type=int, default=1,
                    help="spread3d: also run the 300x300x250 sphere case")
    ap.add_argument("--spread3d-t-mu", type=float, default=50.0,
                    help="spread3d: run length in capillary times")
    ap.add_argument("--shear-t-mu", type=float, default=12.0, help="shear: run length in t_mu")
    ap.add_argument("--case", default="ib-cap", choices=["ib-cap", "batch3d", "batch2d", "step3d"],
                    help="profile: the small case to run (see run_profile_mode)")
    ap.add_argument("--ib-grouped", type=int, default=0, help="profile ib-cap: grouped IB kernels")
    ap.add_argument("--tuning", default="",
                    help="fixed stream-collide launch shape 'variant,block_x,rows,ctas,warps' "
                         "instead of the autotuner (used for profiler runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.mode == "batch":
        return run_batch_mode(args)
    if args.mode == "serve":
        return run_serve_mode(args)
    if args.mode == "shear":
        return run_shear_mode(args)
    if args.mode == "spread2d":
        return run_spread2d_mode(args)
    if args.mode == "spread3d":
        return run_spread3d_mode(args)
    if args.mode == "kernel2d":
        return run_kernel2d_mode(args)
    if args.mode == "profile":
        return run_profile_mode(args)
    from paper_2604_17463_gb300 import workloads as W
    wl = W.drop_3d_256x256x128()
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
