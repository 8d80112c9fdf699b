"""Serving loop and batch runners on top of libiblb's batched engine.

serve():          continuous batching of wetting requests that arrive over
                  time (a Poisson stream): each request is admitted into the
                  D2Q9 or the D3Q19 batch as soon as a slot and arena memory
                  are free (admission and memory are native, in the library);
                  the two batches run on separate CUDA streams so their work
                  overlaps on the device; finished requests are read
                  (observables), released, and their time-to-result recorded.
run_batched():    a fixed set of simulations through one batch.
run_sequential(): the same set one simulation at a time with the single
                  engine (the baseline the batched forms are compared with).
Every step of every simulation runs in the CUDA library.
"""
from __future__ import annotations

import collections
import time
from typing import Dict, List, Optional

import numpy as np

from . import iblb


def _percentile(xs, p):
    return float(np.percentile(np.asarray(xs), p)) if len(xs) else float("nan")


def run_batched(workloads, storage: int, hbm_budget_bytes: int, chunk: int = 2000,
                stream: Optional[int] = None) -> Dict:
    """Run every workload (all of one lattice type) to its step count in one
    batch, admitting more as earlier ones finish.  Returns per-workload
    observables and the wall time."""
    lattice = workloads[0].lattice
    b = iblb.Batch(lattice, storage, hbm_budget_bytes, max_slots=max(64, len(workloads)),
                   stream=stream)
    todo = collections.deque(range(len(workloads)))
    slot_of = {}
    obs = [None] * len(workloads)
    t0 = time.perf_counter()
    while todo or slot_of:
        while todo:
            k = todo[0]
            s = b.admit_workload(workloads[k])
            if s is None:
                break
            slot_of[s] = k
            todo.popleft()
        if not slot_of:
            raise RuntimeError("a workload does not fit in the batch budget")
        b.run(chunk)
        b.sync()
        for s in b.poll():
            k = slot_of.pop(s)
            obs[k] = b.observables(s)
            b.release(s)
    wall = time.perf_counter() - t0
    info = b.info()
    b.close()
    return {"wall_s": wall, "obs": obs, "kernel_launches": info["kernel_launches"]}


def run_sequential(workloads, storage: int, stream: Optional[int] = None) -> Dict:
    """The same workloads one at a time with the single-simulation engine."""
    obs = []
    t0 = time.perf_counter()
    for wl in workloads:
        g = iblb.Simulation.from_workload(wl, storage=storage, stream=stream)
        g.step(wl.steps)
        obs.append(g.observables())
        g.close()
    return {"wall_s": time.perf_counter() - t0, "obs": obs}


def serve(requests, storage: int, budget_2d: int, budget_3d: int, chunk: int = 500,
          max_slots: int = 2048, streams=None) -> Dict:
    """Continuous-batching serving loop over `requests` (workloads.Request,
    arrival times in seconds from the start).  Returns per-request results
    and the throughput / latency summary.  `streams` = (2D, 3D) CUDA stream
    handles; by default two new torch streams."""
    if streams is None:
        import torch

        keep = (torch.cuda.Stream(), torch.cuda.Stream())
        streams = (keep[0].cuda_stream, keep[1].cuda_stream)
    batches = {
        9: iblb.Batch(iblb.D2Q9, storage, budget_2d, max_slots=max_slots, stream=streams[0]),
        19: iblb.Batch(iblb.D3Q19, storage, budget_3d, max_slots=max_slots, stream=streams[1]),
    }
    pending = collections.deque(sorted(range(len(requests)), key=lambda i: requests[i].arrival_s))
    queue: collections.deque = collections.deque()
    inflight = {}
    results: List[Optional[Dict]] = [None] * len(requests)
    max_queue = 0
    t0 = time.perf_counter()
    while pending or queue or inflight:
        now = time.perf_counter() - t0
        while pending and requests[pending[0]].arrival_s <= now:
            queue.append(pending.popleft())
        # admission: every queued request that fits now (first come, first
        # tried; a large one that does not fit does not block smaller ones)
        keep = collections.deque()
        for i in queue:
            wl = requests[i].work
            s = batches[wl.lattice].admit_workload(wl)
            if s is None:
                keep.append(i)
            else:
                inflight[(wl.lattice, s)] = i
                results[i] = {"admitted_s": time.perf_counter() - t0}
        queue = keep
        max_queue = max(max_queue, len(queue))
        if not inflight:
            if pending:
                time.sleep(max(0.0, requests[pending[0]].arrival_s - (time.perf_counter() - t0)))
            continue
        # both batches advance concurrently on their own streams, each by at
        # most `chunk` steps and never past its next completion, so that a
        # finished request is read and its room freed in the same round
        for b in batches.values():
            left = b.steps_to_next_completion()
            if left > 0:
                b.run(min(chunk, left))
        for b in batches.values():
            b.sync()
        for lat, b in batches.items():
            for s in b.poll():
                i = inflight.pop((lat, s))
                o = b.observables(s)
                b.release(s)
                t_done = time.perf_counter() - t0
                r = requests[i]
                results[i].update({"done_s": t_done, "latency_s": t_done - r.arrival_s,
                                   "theta_deg": o["theta_deg"], "volume": o["volume"],
                                   "height": o["height"],
                                   "name": r.work.name, "lattice": r.work.lattice,
                                   "cells": r.work.cells, "steps": r.work.steps})
    wall = time.perf_counter() - t0
    launches = sum(b.info()["kernel_launches"] for b in batches.values())
    for b in batches.values():
        b.close()
    lat = [r["latency_s"] for r in results if r is not None]
    updates = sum(r["cells"] * r["steps"] for r in results if r is not None)
    return {
        "results": results,
        "wall_s": wall,
        "completed": len(lat),
        "sims_per_hour": len(lat) / wall * 3600.0,
        "p50_s": _percentile(lat, 50),
        "p99_s": _percentile(lat, 99),
        "mlups": updates / wall / 1e6,
        "max_queue": max_queue,
        "kernel_launches": launches,
    }
