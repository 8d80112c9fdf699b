"""Batched engine: many simulations of uneven size advanced by shared launches.

Each slot must give the same result as the same simulation run alone (single
engine, or alone in a batch), within the stated tolerance of its storage:
FP64 1e-10 (also against the oracle), FP32 1e-5 relative L2 on u; binary16
storage is compared on u with 1e-3 and on the contact angle with 0.1 deg.
"""
import math

import numpy as np
import pytest

from paper_2604_17463_gb300 import iblb
from paper_2604_17463_gb300 import workloads as W
from helpers import fluid_mask, oracle_from_workload, rel_l2

pytestmark = pytest.mark.gpu

GB = 1 << 30


def drops_2d():
    # ragged widths, different angles and relaxation times
    return [W.droplet_2d(w, th, tau, 100, name=f"b{i}")
            for i, (w, th, tau) in enumerate([(67, 45.0, 0.7), (100, 120.0, 1.3),
                                              (129, 80.0, 0.9), (256, 60.0, 1.0)])]


def single(wl, storage, steps):
    g = iblb.Simulation.from_workload(wl, storage=storage)
    g.step(steps)
    rho, u, q = g.fields()
    o = g.observables()
    g.close()
    return rho, u, q, o


@pytest.mark.parametrize("storage,tol", [(iblb.FP64, 1e-10), (iblb.FP32_DEV, 1e-5)])
def test_batch_slots_match_single_engine(storage, tol):
    steps = 300
    wls = drops_2d()
    b = iblb.Batch(iblb.D2Q9, storage, 1 * GB, max_slots=16)
    slots = [b.admit_workload(wl, n_steps=steps) for wl in wls]
    assert all(s is not None for s in slots)
    done = b.run(steps + 50)
    assert done == len(wls)
    assert sorted(b.poll()) == sorted(slots)
    for wl, s in zip(wls, slots):
        assert b.steps_done(s) == steps
        rho_b, u_b, q_b = b.fields(s)
        rho_s, u_s, q_s, o_s = single(wl, storage, steps)
        m = fluid_mask(rho_s.shape, 2)
        assert rel_l2(u_b[:, m], u_s[:, m]) < tol
        assert rel_l2(rho_b[m] - 1, rho_s[m] - 1) < 10 * tol
        # node positions: FP64 agrees to round-off, FP32 to its own rounding
        assert np.max(np.abs(q_b - q_s)) < (1e-11 if storage == iblb.FP64 else 1e-6)
        o_b = b.observables(s)
        assert abs(o_b["volume"] - o_s["volume"]) < 1e-8 * abs(o_s["volume"])
    b.close()


def test_batch_fp64_slot_matches_oracle():
    wl = drops_2d()[0]
    b = iblb.Batch(iblb.D2Q9, iblb.FP64, 1 * GB, max_slots=4)
    others = [b.admit_workload(w, n_steps=150) for w in drops_2d()[1:]]
    s = b.admit_workload(wl, n_steps=200)
    assert s is not None and all(o is not None for o in others)
    b.run(200)
    rho_b, u_b, q_b = b.fields(s)
    o = oracle_from_workload(wl)
    assert o.step(200) == 0
    ro, uo, qo = o.fields()
    m = fluid_mask(ro.shape, 2)
    assert rel_l2(u_b[:, m], uo[:2, m]) < 1e-10
    assert rel_l2(rho_b[m], ro[m]) < 1e-12
    assert np.max(np.abs(q_b - qo)) < 1e-11
    b.close()


@pytest.mark.parametrize("storage,tol", [(iblb.FP32_DEV, 1e-5), (iblb.FP16_DEV, 1e-3)])
def test_same_result_alone_and_in_the_mix(storage, tol):
    steps = 400
    target = W.droplet_2d(96, 70.0, 0.8, steps, name="target")
    alone = iblb.Batch(iblb.D2Q9, storage, 1 * GB, max_slots=4)
    sa = alone.admit_workload(target, n_steps=steps)
    alone.run(steps)
    ua = alone.fields(sa)[1]
    oa = alone.observables(sa)
    mix = iblb.Batch(iblb.D2Q9, storage, 1 * GB, max_slots=32)
    rng = np.random.default_rng(5)
    for k in range(12):   # others of different sizes and step counts
        w = int(rng.integers(64, 400))
        mix.admit_workload(W.droplet_2d(w, float(rng.uniform(30, 150)), float(rng.uniform(0.6, 1.4)),
                                        0), n_steps=int(rng.integers(100, 700)))
    sm = mix.admit_workload(target, n_steps=steps)
    # more arrivals while it runs
    mix.run(150)
    for k in range(4):
        mix.admit_workload(W.droplet_2d(int(rng.integers(64, 300)), 90.0, 1.0, 0), n_steps=300)
    mix.run(1000)
    assert mix.steps_done(sm) == steps
    um = mix.fields(sm)[1]
    om = mix.observables(sm)
    m = fluid_mask(um.shape[1:], 2)
    assert rel_l2(um[:, m], ua[:, m]) < tol
    assert abs(om["theta_deg"] - oa["theta_deg"]) < 0.1
    alone.close()
    mix.close()


def test_admission_budget_release_and_eagain():
    wl = W.droplet_2d(512, 60.0, 1.0, 0)
    cfg = iblb.make_config(9, wl.nx, wl.ny, storage=iblb.FP32_DEV, xi=wl.xi, theta_eq_deg=60.0)
    fp = iblb.Batch.footprint(cfg, wl.nodes.shape[0])
    b = iblb.Batch(iblb.D2Q9, iblb.FP32_DEV, int(2.5 * fp), max_slots=8)
    s0 = b.admit(cfg, wl.nodes, n_steps=10)
    s1 = b.admit(cfg, wl.nodes, n_steps=20)
    assert s0 is not None and s1 is not None
    assert b.admit(cfg, wl.nodes, n_steps=10) is None        # no room: EAGAIN
    free_before = b.info()["free_bytes"]
    assert b.run(10) == 1
    assert b.poll() == [s0]
    b.release(s0)
    assert b.info()["free_bytes"] >= free_before + fp - 512
    s2 = b.admit(cfg, wl.nodes, n_steps=5)                     # room again
    assert s2 is not None
    assert b.run(100) == 2
    assert sorted(b.poll()) == sorted([s1, s2])
    assert b.steps_done(s1) == 20 and b.steps_done(s2) == 5
    b.close()


def test_batch_3d_slots_match_single_engine():
    steps = 60
    wls = [W.droplet_3d(64, 64, 48, 75.0, 0.8, steps, name="a"),
           W.droplet_3d(96, 80, 40, 110.0, 1.1, steps, name="b")]
    b = iblb.Batch(iblb.D3Q19, iblb.FP32_DEV, 2 * GB, max_slots=4)
    slots = [b.admit_workload(wl, n_steps=steps) for wl in wls]
    assert b.run(steps) == 2
    for wl, s in zip(wls, slots):
        rho_b, u_b, q_b = b.fields(s)
        rho_s, u_s, q_s, _ = single(wl, iblb.FP32_DEV, steps)
        m = fluid_mask(rho_s.shape, 3)
        assert rel_l2(u_b[:, m], u_s[:, m]) < 1e-5
        assert np.max(np.abs(q_b - q_s)) < 1e-7
        assert b.tile(s) in (2, 4, 8, 16)
    b.close()


def test_invalid_requests_are_refused():
    b = iblb.Batch(iblb.D2Q9, iblb.FP32_DEV, 64 << 20, max_slots=2)
    wl = W.droplet_2d(64, 60.0, 1.0, 0)
    bad = iblb.make_config(19, 64, 16, 16, storage=iblb.FP32_DEV)   # wrong lattice
    with pytest.raises(iblb.IBLBError):
        b.admit(bad, wl.nodes, n_steps=5)
    cfg = iblb.make_config(9, 64, 16, storage=iblb.FP32_DEV, xi=wl.xi)
    sunk = wl.nodes.copy()
    sunk[:, 1] -= 20.0
    with pytest.raises(iblb.IBLBError) as e:
        b.admit(cfg, sunk, n_steps=5)
    assert e.value.status == 4
    b.close()
