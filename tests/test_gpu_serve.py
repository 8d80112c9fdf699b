"""Serving loop: continuous batching of wetting requests that arrive over
time; every request completes, and its result equals the same request run
alone through the single-simulation engine (same storage), within the FP32
tolerance on the contact angle and volume."""
import numpy as np
import pytest

from paper_2604_17463_gb300 import iblb, serve
from paper_2604_17463_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_serving_completes_and_matches_alone():
    reqs = W.serve_requests(count=24, rate_per_s=60.0, steps_lo=200, steps_hi=800, frac_3d=0.2)
    out = serve.serve(reqs, iblb.FP32_DEV, budget_2d=2 << 30, budget_3d=8 << 30, chunk=200)
    assert out["completed"] == len(reqs)
    assert out["p99_s"] >= out["p50_s"] > 0
    # a sample of requests run alone
    for i in range(0, len(reqs), 6):
        wl = reqs[i].work
        g = iblb.Simulation.from_workload(wl, storage=iblb.FP32_DEV)
        g.step(wl.steps)
        o = g.observables()
        g.close()
        r = out["results"][i]
        if np.isfinite(o["theta_deg"]):
            assert abs(r["theta_deg"] - o["theta_deg"]) < 0.1
        assert abs(r["volume"] / o["volume"] - 1) < 1e-5


def test_small_budget_queues_requests():
    # identical requests that all arrive at once, with a budget for two: the
    # others wait in the queue and are admitted as slots finish
    wl = W.droplet_2d(256, 60.0, 1.0, 200, name="q")
    reqs = [W.Request(0.0, wl) for _ in range(6)]
    fp = iblb.Batch.footprint(iblb.make_config(9, wl.nx, wl.ny, storage=iblb.FP32_DEV),
                              wl.nodes.shape[0])
    out = serve.serve(reqs, iblb.FP32_DEV, budget_2d=int(2.5 * fp), budget_3d=1 << 20, chunk=50)
    assert out["completed"] == len(reqs)
    assert out["max_queue"] >= 4
    done = sorted(r["done_s"] for r in out["results"])
    # completions come in waves of two
    assert done[2] > done[1] and done[4] > done[3]
