"""The pipelined stream-collide kernel (bulk asynchronous copies into shared
memory, persistent CTAs) against the plain kernel and against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import iblb
from paper_2604_17463_gb300 import workloads as W
from helpers import fluid_mask, oracle_from_workload, rel_l2

pytestmark = pytest.mark.gpu


def near_eq(Q, shape, seed, amp=0.03):
    _, w, _ = oracle.lattice(Q)
    return w.reshape((Q,) + (1,) * len(shape)) * (1.0 + W.random_perturbation((Q,) + shape, seed, amp))


CASES = [
    (9, (256, 10, 1), True),      # rows mode, bounce-back rows inside a tile
    (9, (96, 13, 1), True),       # rows mode, narrow rows, ragged last tile
    (9, (2048, 6, 1), True),      # segment mode: two 1024-cell tiles per row
    (9, (512, 7, 1), False),      # periodic along every axis
    (19, (256, 5, 6), True),      # D3Q19, fewer tiles than CTAs
    (19, (64, 7, 5), True),       # D3Q19, y seam inside a tile
    (19, (2048, 3, 4), False),    # D3Q19 segment mode, periodic
]


@pytest.mark.parametrize("Q,dims,walls", CASES)
@pytest.mark.parametrize("storage", [iblb.FP64, iblb.FP32_DEV, iblb.FP16_DEV])
def test_pipeline_matches_plain_and_oracle(Q, dims, walls, storage):
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    body = (2e-6, -1e-6, 5e-7 if Q == 19 else 0.0)
    f0 = near_eq(Q, shape, seed=nx + ny)
    sims = []
    for variant in (0, 1):
        g = iblb.Simulation(Q, nx, ny, nz, tau=0.83, walls=walls, wetting=False, body_force=body,
                            storage=storage)
        g.set_tuning(variant, rows_per_tile=3)
        # wide FP64 rows leave no room for a 2-stage pipeline: plain fallback
        assert g.variant == variant or (variant == 1 and storage == iblb.FP64)
        g.set_populations(f0)
        g.step(4)
        sims.append(g)
    fa, fb = sims[0].populations(), sims[1].populations()
    m = fluid_mask(shape, 2 if Q == 9 else 3, walls)
    # identical arithmetic: agreement to the last bits of the storage format
    tol = {iblb.FP64: 1e-15, iblb.FP32_DEV: 1e-7, iblb.FP16_DEV: 1e-6}[storage]
    assert np.max(np.abs(fa[:, m] - fb[:, m])) < tol
    if storage == iblb.FP64:
        o = oracle.Sim(Q, nx, ny, nz, tau=0.83, walls=walls, wetting=False, body_force=body)
        o.set_populations(f0)
        o.step(4)
        assert np.max(np.abs(fb[:, m] - o.populations()[:, m])) < 1e-14
    for g in sims:
        g.close()


@pytest.mark.parametrize("storage,tol", [(iblb.FP64, 1e-10), (iblb.FP32_DEV, 1e-5)])
def test_pipeline_full_step_3d_drop(storage, tol):
    # a drop on a lattice whose width selects the pipelined kernel
    R, xi = 6.0, 1.0
    nodes, faces = W.icosphere(2, R, (128.3, 9.7, W.WALL_PLANE + R + 2 * xi))
    wl = W.Workload("pipe3d", 19, 256, 20, 18, 0.8, 5e-3, xi, 75.0, 9, 3, 10, nodes, faces)
    o = oracle_from_workload(wl)
    g = iblb.Simulation.from_workload(wl, storage=storage)
    assert g.variant == 1
    o.step(8)
    g.step(8)
    ro, uo, qo = o.fields()
    rg, ug, qg = g.fields()
    m = fluid_mask(o.shape, 3)
    assert rel_l2(ug[:, m], uo[:, m]) < tol
    assert rel_l2(rg[m], ro[m]) < tol
    g.close()


def test_pipeline_used_by_default_on_benchmark_shape():
    wl = W.config3()
    g = iblb.Simulation.from_workload(wl, storage=iblb.FP32_DEV)
    assert g.variant == 1
    g.step(3)
    g.sync()
    g.close()


def test_autotune_leaves_state_unchanged():
    R, xi = 6.0, 1.0
    nodes, faces = W.icosphere(2, R, (64.3, 9.7, W.WALL_PLANE + R + 2 * xi))
    wl = W.Workload("tune3d", 19, 128, 20, 18, 0.8, 5e-3, xi, 75.0, 9, 3, 10, nodes, faces)
    a = iblb.Simulation.from_workload(wl, storage=iblb.FP32_DEV)
    b = iblb.Simulation.from_workload(wl, storage=iblb.FP32_DEV)
    a.step(5)
    b.step(5)
    pick = b.autotune(trials=3)
    assert pick["variant"] in (0, 1)
    a.step(5)
    b.step(5)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fa - fb)) < 1e-7
    _, _, qa = a.fields()
    _, _, qb = b.fields()
    assert np.max(np.abs(qa - qb)) < 1e-9
    a.close()
    b.close()
