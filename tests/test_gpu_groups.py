"""Grouped spreading and interpolation of 3D interfaces (Eq. 7-8, tuning
ib_grouped = 1): the nodes of one 8 x 8 x 8 lattice tile form a group, whose
stencils are summed in (or read from) a box of the lattice in shared memory.

Checked against the FP64 oracle and against the per-node kernels (the
default):
- the force field and the band flags it leaves (FP64 to 1e-13, FP32 to 1e-6
  of the largest component);
- the interpolated velocity;
- full steps across several 32-step regroup chunks.

The cases are:
- drops across the periodic seams;
- a fully periodic box;
- a dense mesh with several groups per tile;
- a strong shear that moves nodes across tiles between regroups;
- nodes above the top wall, whose groups' boxes are too large for shared
  memory and take the per-node fallback.
"""
import dataclasses

import numpy as np
import pytest

from paper_2604_17463_gb300 import iblb
from paper_2604_17463_gb300 import workloads as W
from helpers import fluid_mask, oracle_from_workload, rel_l2, small_3d

pytestmark = pytest.mark.gpu


def seam_3d():
    wl = small_3d(n=22, nz=17, R=5.0)
    wl.nodes = wl.nodes.copy()
    wl.nodes[:, 0] -= 10.6
    wl.nodes[:, 1] += 9.7
    return wl


def periodic_3d():
    wl = small_3d(n=20, nz=18, R=5.0)
    return dataclasses.replace(wl, walls=False, wetting=False, nodes=wl.nodes + [0.0, 0.0, 1.3])


def dense_3d():
    # 10 242 nodes on a radius-11 sphere: ~6.7 nodes per unit area, so a tile
    # holds several 128-node groups
    nodes, faces = W.icosphere(5, 11.0, (20.0 + 0.31, 20.0 - 0.22, W.WALL_PLANE + 11.0 + 2.0))
    return W.Workload("dense3d", 19, 40, 40, 30, 0.8, 5e-3, 1.0, 75.0, 9, 3, 100, nodes, faces)


def above_top_3d():
    # the top cap of the drop pushed through the upper wall: stencil points
    # at or beyond the top solid layer take no force, and the groups with
    # such nodes have boxes too tall for shared memory
    wl = small_3d(n=24, nz=16, R=6.0)
    q = wl.nodes.copy()
    top = q[:, 2] > q[:, 2].max() - 2.5
    q[top, 2] += 14.0
    return dataclasses.replace(wl, nodes=q)


CASES = {"3d": small_3d, "3d_seam": seam_3d, "3d_periodic": periodic_3d, "3d_dense": dense_3d,
         "3d_above_top": above_top_3d}


@pytest.mark.parametrize("which", list(CASES))
@pytest.mark.parametrize("storage,tol", [(iblb.FP64, 1e-13), (iblb.FP32_DEV, 1e-6)])
def test_force_field_grouped(which, storage, tol):
    wl = CASES[which]()
    o = oracle_from_workload(wl)
    Fo, bad = o.force_field()
    g = iblb.Simulation.from_workload(wl, storage=storage)
    a = iblb.Simulation.from_workload(wl, storage=storage)
    g.set_tuning(0, 128, ib_grouped=1)
    assert g.tuning()["ib_grouped"] == 1 and a.tuning()["ib_grouped"] == 0
    Fg, Fa = g.force_field(), a.force_field()
    scale = np.max(np.abs(Fo[:3]))
    assert scale > 0
    assert np.max(np.abs(Fg - Fo[:3])) <= tol * scale
    assert np.max(np.abs(Fg - Fa)) <= tol * scale
    # the force buffer and the flags are left cleared: the same field again
    F2 = g.force_field()
    assert np.max(np.abs(F2 - Fg)) <= tol * scale
    g.close()
    a.close()


@pytest.mark.parametrize("which", list(CASES))
@pytest.mark.parametrize("storage,tol", [(iblb.FP64, 1e-13), (iblb.FP32_DEV, 2e-6)])
def test_interpolate_grouped(which, storage, tol):
    wl = CASES[which]()
    o = oracle_from_workload(wl)
    g = iblb.Simulation.from_workload(wl, storage=storage)
    g.set_tuning(0, 128, ib_grouped=1)
    rng = np.random.default_rng(77)
    u = rng.normal(size=(3,) + o.shape) * 1e-3
    qo = o.interpolate(u)
    qg = g.interpolate(u)
    assert np.max(np.abs(qg - qo)) <= 1e-17 + tol * np.max(np.abs(qo))
    g.close()


@pytest.mark.parametrize("which,steps", [("3d_dense", 40), ("3d_seam", 70), ("3d_periodic", 40)])
def test_full_step_grouped_fp64(which, steps):
    # more than one 32-step chunk: the groups are rebuilt from moved nodes
    wl = CASES[which]()
    o = oracle_from_workload(wl)
    g = iblb.Simulation.from_workload(wl)
    g.set_tuning(0, 128, ib_grouped=1)
    assert o.step(steps) == 0
    g.step(steps)
    ro, uo, qo = o.fields()
    rg, ug, qg = g.fields()
    m = fluid_mask(o.shape, 3, wl.walls)
    assert rel_l2(rg[m] - 1.0, ro[m] - 1.0) < 1e-10
    assert rel_l2(ug[:, m], uo[:, m]) < 1e-10
    assert np.max(np.abs(qg - qo)) < 1e-11
    g.close()


def shear_u(shape, rate):
    nz, ny, nx = shape
    u = np.zeros((3,) + shape)
    z = np.arange(nz, dtype=float)[:, None, None]
    u[0] = rate * (z - nz / 2.0) * np.ones(shape)
    u[1] = 0.5 * rate * (z - nz / 2.0) * np.ones(shape)
    return u


def test_strong_shear_moves_nodes_between_regroups():
    # u_x differs by ~0.1 across a tile: nodes of a group drift ~3 cells
    # apart within a 32-step chunk, so boxes grow past a tile (some beyond
    # the FP64 capacity) before the next regroup
    wl = small_3d(n=32, nz=24, R=7.0, level=3)
    steps = 70
    o = oracle_from_workload(wl)
    g = iblb.Simulation.from_workload(wl)
    g.set_tuning(0, 128, ib_grouped=1)
    u = shear_u(o.shape, 0.012)
    o.set_equilibrium(u)
    g.set_equilibrium(u)
    assert o.step(steps) == 0
    g.step(steps)
    ro, uo, qo = o.fields()
    rg, ug, qg = g.fields()
    m = fluid_mask(o.shape, 3)
    assert rel_l2(ug[:, m], uo[:, m]) < 1e-10
    assert np.max(np.abs(qg - qo)) < 1e-11
    q0 = wl.nodes
    assert np.max(np.abs(qo[:, 0] - q0[:, 0])) > 3.0  # the nodes did move
    g.close()


@pytest.mark.parametrize("storage", [iblb.FP32_DEV, iblb.FP16_DEV])
def test_grouped_matches_per_node_reduced_precision(storage):
    wl = dense_3d()
    steps = 70
    g = iblb.Simulation.from_workload(wl, storage=storage)
    a = iblb.Simulation.from_workload(wl, storage=storage)
    a.set_tuning(0, 128)
    g.set_tuning(0, 128, ib_grouped=1)
    g.step(steps)
    a.step(steps)
    rg, ug, qg = g.fields()
    ra, ua, qa = a.fields()
    m = fluid_mask(rg.shape, 3)
    # binary16: a different order of the FP32 force additions changes the
    # stochastically rounded bits, and the runs drift apart by ~1e-3 of u
    tol, qtol = (1e-5, 1e-6) if storage == iblb.FP32_DEV else (1e-3, 2e-5)
    assert rel_l2(ug[:, m], ua[:, m]) < tol
    assert np.max(np.abs(qg - qa)) < qtol
    g.close()
    a.close()


def test_autotune_keeps_the_ib_choice():
    wl = small_3d()
    g = iblb.Simulation.from_workload(wl, storage=iblb.FP32_DEV)
    g.set_tuning(0, 128, ib_grouped=1)
    t = g.autotune(trials=2)
    assert t["ib_grouped"] == 1 and g.tuning()["ib_grouped"] == 1
    g.close()
