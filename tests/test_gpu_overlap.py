"""The overlapped time step (iblb_tuning.step_overlap): stream-collide of
every cell with the body force only on one stream while the nodal forces are
computed and spread on another, then the flagged band cells updated again
with their force density.

The band cells take the same arithmetic as in one pass, so with the ordered
(deterministic) spread the overlapped and the serial step give bitwise the
same fields and nodes in every storage form, kernel variant, lattice and wall
condition; with the atomic spread they agree to the storage tolerance, and
the FP64 run matches the oracle.  Runs cross the 32-step graph chunks and end
with the step that writes every cell's moments.
"""
import numpy as np
import pytest

from paper_2604_17463_gb300 import iblb
from paper_2604_17463_gb300 import workloads as W
from helpers import fluid_mask, oracle_from_workload, rel_l2, small_2d, small_3d

pytestmark = pytest.mark.gpu


def run(wl, storage, overlap, variant=0, block_x=128, steps=45, det=True, **over):
    g = iblb.Simulation.from_workload(wl, storage=storage, deterministic_spread=det, **over)
    g.set_tuning(variant, block_x, step_overlap=overlap)
    g.step(steps)
    out = g.fields()
    g.close()
    return out


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("which", ["2d", "3d"])
@pytest.mark.parametrize("storage", [iblb.FP64, iblb.FP32_DEV, iblb.FP16_DEV])
def test_overlapped_equals_serial_bitwise(which, storage):
    wl = small_2d(nx=64, ny=40) if which == "2d" else small_3d()
    a = run(wl, storage, overlap=1)
    b = run(wl, storage, overlap=2)
    assert same(a, b)


@pytest.mark.parametrize("variant,block_x", [(0, 64), (0, 256), (2, 128), (3, 128), (1, 128)])
@pytest.mark.parametrize("storage", [iblb.FP32_DEV, iblb.FP16_DEV])
def test_overlapped_bulk_variants_3d(variant, block_x, storage):
    # each stream-collide variant as the bulk pass, against the serial plain
    # kernel (the variants agree to FP32 rounding, binary16 to its rounding)
    wl = small_3d(n=32, nz=20)
    a = run(wl, storage, overlap=1, variant=variant, block_x=block_x)
    b = run(wl, storage, overlap=2, variant=0, block_x=128)
    m = fluid_mask(a[0].shape, 3)
    tol, qtol = (1e-5, 1e-6) if storage == iblb.FP32_DEV else (2e-3, 2e-5)
    assert rel_l2(a[1][:, m], b[1][:, m]) < tol
    assert np.max(np.abs(a[2] - b[2])) < qtol


@pytest.mark.parametrize("variant", [0, 2, 1])
def test_overlapped_bulk_variants_2d(variant):
    wl = small_2d(nx=128, ny=48, R=9.0)
    a = run(wl, iblb.FP32_DEV, overlap=1, variant=variant)
    b = run(wl, iblb.FP32_DEV, overlap=2)
    m = fluid_mask(a[0].shape, 2)
    assert rel_l2(a[1][:, m], b[1][:, m]) < 1e-5


@pytest.mark.parametrize("which,steps", [("2d", 70), ("3d", 40)])
def test_overlapped_atomic_spread_matches_oracle(which, steps):
    wl = small_2d(nx=64, ny=40) if which == "2d" else small_3d()
    g = iblb.Simulation.from_workload(wl)
    g.set_tuning(0, 128, step_overlap=1)
    g.step(steps)
    rg, ug, qg = g.fields()
    o = oracle_from_workload(wl)
    assert o.step(steps) == 0
    ro, uo, qo = o.fields()
    m = fluid_mask(o.shape, wl.dim)
    assert rel_l2(rg[m] - 1.0, ro[m] - 1.0) < 1e-10
    assert rel_l2(ug[:, m], uo[: wl.dim, m]) < 1e-10
    assert np.max(np.abs(qg - qo)) < 1e-11
    g.close()


@pytest.mark.parametrize("storage", [iblb.FP64, iblb.FP32_DEV, iblb.FP16_DEV])
def test_overlapped_atomic_spread_bitwise_when_stencils_are_disjoint(storage):
    # with nodes 9.5 cells apart no two stencils share a cell, so the atomic
    # spread's sums are exact and the overlapped and serial steps agree
    # bitwise
    nodes, faces = W.icosphere(0, 9.0, (16.3, 15.8, W.WALL_PLANE + 12.0))
    wl = W.Workload("sparse3d", 19, 32, 32, 28, 0.8, 5e-3, 1.0, 75.0, 9, 3, 40, nodes, faces)
    a = run(wl, storage, overlap=1, det=False)
    b = run(wl, storage, overlap=2, det=False)
    assert same(a, b)


@pytest.mark.parametrize("storage,tol", [(iblb.FP64, 1e-12), (iblb.FP32_DEV, 1e-5)])
def test_overlapped_atomic_spread_matches_serial(storage, tol):
    wl = small_3d(n=30, nz=22, R=7.0, level=3)
    a = run(wl, storage, overlap=1, det=False, steps=70)
    b = run(wl, storage, overlap=2, det=False, steps=70)
    m = fluid_mask(a[0].shape, 3)
    assert rel_l2(a[1][:, m], b[1][:, m]) < tol
    assert np.max(np.abs(a[2] - b[2])) < tol


def test_overlapped_moving_walls_bitwise():
    wl = small_3d(n=28, nz=22)
    kw = dict(wall_u_lo=(-0.01, 0.0, 0.0), wall_u_hi=(0.01, 0.004, 0.0))
    a = run(wl, iblb.FP64, overlap=1, **kw)
    b = run(wl, iblb.FP64, overlap=2, **kw)
    assert same(a, b)


def test_overlapped_single_steps_and_profiled_mix():
    # one-step calls (each its own graph, each writing every moment) and a
    # profiled (serial) step in between: the same as one serial run
    wl = small_3d()
    g = iblb.Simulation.from_workload(wl, storage=iblb.FP32_DEV, deterministic_spread=True)
    g.set_tuning(0, 128, step_overlap=1)
    for _ in range(5):
        g.step(1)
    g.step_profiled(3)
    g.step(33)
    a = g.fields()
    g.close()
    b = run(wl, iblb.FP32_DEV, overlap=2, steps=41)
    assert same(a, b)


def test_overlap_setting_round_trips_and_is_validated():
    g = iblb.Simulation.from_workload(small_3d(), storage=iblb.FP32_DEV)
    assert g.tuning()["step_overlap"] == 0
    g.set_tuning(0, 64, step_overlap=2)
    assert g.tuning()["step_overlap"] == 2
    assert g.autotune(trials=1)["step_overlap"] == 2
    with pytest.raises(iblb.IBLBError):
        g.set_tuning(0, 64, step_overlap=3)
    g.close()
