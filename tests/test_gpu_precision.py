"""Reduced-precision population storage against FP64 on a spreading drop.

Workload: the 4x-downscaled copy of the 2D spreading configuration
(512 x 128 D2Q9, R = 50 with 500 nodes, initial angle 150 deg, theta_eq = 60
deg, tau = 1).  The FP64 GPU run is checked against the oracle on the first
steps; FP32 and binary16 deviation storage are checked against the FP64 GPU
run on the apparent contact angle (0.1 deg), the contact-line radius and the
film thickness along the whole run.
"""
import math

import numpy as np
import pytest

from paper_2604_17463_gb300 import iblb
from paper_2604_17463_gb300 import workloads as W
from helpers import fluid_mask, oracle_from_workload, rel_l2

pytestmark = pytest.mark.gpu

CHECKPOINTS = 8
STEPS_PER = 10000   # 80k steps, about 10 viscous times mu R / sigma


def trajectory(wl, storage):
    g = iblb.Simulation.from_workload(wl, storage=storage)
    out = []
    for _ in range(CHECKPOINTS):
        g.step(STEPS_PER)
        out.append(g.observables())
    g.close()
    return out


@pytest.fixture(scope="module")
def runs():
    wl = W.spreading_2d_2048x512(theta_eq_deg=60.0, tau=1.0, downscale=4)
    return {s: trajectory(wl, s) for s in (iblb.FP64, iblb.FP32_DEV, iblb.FP16_DEV)}


def test_fp64_matches_oracle_on_downscaled_spreading():
    wl = W.spreading_2d_2048x512(theta_eq_deg=60.0, tau=1.0, downscale=4)
    o = oracle_from_workload(wl)
    g = iblb.Simulation.from_workload(wl)
    assert o.step(300) == 0
    g.step(300)
    ro, uo, qo = o.fields()
    rg, ug, qg = g.fields()
    m = fluid_mask(o.shape, 2)
    assert rel_l2(rg[m], ro[m]) < 1e-10
    assert rel_l2(ug[:, m], uo[:2, m]) < 1e-10
    oo, og = o.observables(), g.observables()
    assert abs(oo["theta_deg"] - og["theta_deg"]) < 1e-8
    g.close()


@pytest.mark.parametrize("storage", [iblb.FP32_DEV, iblb.FP16_DEV])
def test_reduced_precision_contact_angle(runs, storage):
    ref = runs[iblb.FP64]
    got = runs[storage]
    worst = max(abs(a["theta_deg"] - b["theta_deg"]) for a, b in zip(got, ref))
    print(f"storage {storage}: max |d theta| = {worst:.4f} deg over "
          f"{CHECKPOINTS * STEPS_PER} steps; final theta {got[-1]['theta_deg']:.3f} "
          f"vs {ref[-1]['theta_deg']:.3f}")
    assert worst < 0.1
    for a, b in zip(got, ref):
        assert abs(a["r_cl"] - b["r_cl"]) < 0.05 * max(b["r_cl"], 1.0)
        assert abs(a["film"] - b["film"]) < 0.01 * wl_xi()
        assert abs(a["volume"] / b["volume"] - 1) < 1e-3
    # the drop really spread (the comparison is not of a frozen state)
    assert ref[-1]["theta_deg"] < ref[0]["theta_deg"] - 10.0


def wl_xi():
    return W.spreading_2d_2048x512(downscale=4).xi


def test_full_size_spreading_fp16_vs_fp64():
    # the full 2048 x 512 spreading drop, the most-spreading corner of the
    # sweep (theta_eq = 30 deg, tau = 0.6), all 200k steps
    wl = W.spreading_2d_2048x512(theta_eq_deg=30.0, tau=0.6)
    runs = {}
    for st in (iblb.FP64, iblb.FP16_DEV):
        g = iblb.Simulation.from_workload(wl, storage=st)
        out = []
        for _ in range(10):
            g.step(wl.steps // 10)
            out.append(g.observables())
        g.close()
        runs[st] = out
    worst = max(abs(a["theta_deg"] - b["theta_deg"])
                for a, b in zip(runs[iblb.FP16_DEV], runs[iblb.FP64]))
    print(f"2048x512 theta_eq 30 tau 0.6: max |d theta| fp16 vs fp64 = {worst:.4f} deg; "
          f"final {runs[iblb.FP16_DEV][-1]['theta_deg']:.2f} deg")
    assert worst < 0.1
    assert runs[iblb.FP64][-1]["theta_deg"] < 100.0
