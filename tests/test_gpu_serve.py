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
    reqs = W.config5(count=24, rate_per_s=60.0, steps_lo=200, steps_hi=800, frac_3d=0.2)
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
    # a budget that holds only a few requests at a time: the rest wait in the
    # queue and are admitted as slots finish
    reqs = W.config5(count=12, rate_per_s=1000.0, steps_lo=100, steps_hi=300, frac_3d=0.0)
    big = max(iblb.Batch.footprint(iblb.make_config(9, r.work.nx, r.work.ny, storage=iblb.FP32_DEV),
                                   r.work.nodes.shape[0]) for r in reqs)
    out = serve.serve(reqs, iblb.FP32_DEV, budget_2d=3 * big, budget_3d=1 << 20, chunk=50)
    assert out["completed"] == len(reqs)
    assert out["max_queue"] > 0
