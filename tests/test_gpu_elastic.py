"""Elastic interface (Skalak strain energy, iblb_config.shear_modulus /
skalak_c) on the GPU against the FP64 oracle.

Per kernel: the nodal forces of a deformed interface equal the oracle's
tension + wetting force plus its elastic force relative to the interface as
set, to 1e-13 relative.  Full step: a capsule deformed by an imposed shear
flow matches the oracle within the FP64 tolerances (relative L2 <= 1e-10 on
rho - 1 and u, nodes to 1e-11), and FP32 storage within 1e-5.  A batched
slot matches the single engine.
"""
import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import iblb
from helpers import fluid_mask, oracle_from_workload, rel_l2, small_2d, small_3d

pytestmark = pytest.mark.gpu

GB = 1 << 30
ELASTIC = dict(shear_modulus=4e-3, skalak_c=1.0)


def shear_field(shape, dim, rate):
    """u_x = rate (a - a_mid) along the wall axis a: a flow that stretches and
    tilts the drop."""
    nz, ny, nx = shape
    u = np.zeros((dim,) + shape)
    if dim == 2:
        a = np.arange(ny, dtype=float)[None, :, None]
        u[0] = rate * (a - ny / 2.0) * np.ones(shape)
    else:
        a = np.arange(nz, dtype=float)[:, None, None]
        u[0] = rate * (a - nz / 2.0) * np.ones(shape)
    return u


def pair(wl, storage, **kw):
    o = oracle_from_workload(wl, **ELASTIC)
    g = iblb.Simulation.from_workload(wl, storage=storage, **ELASTIC, **kw)
    u = shear_field(o.shape, wl.dim, 2e-3)
    o.set_equilibrium(u)
    g.set_equilibrium(u)
    return o, g


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_nodal_forces_of_a_deformed_interface(which):
    wl = small_2d() if which == "2d" else small_3d()
    _, g = pair(wl, iblb.FP64)
    g.step(30)
    q = g.fields()[2]
    pg, ng, cg = g.nodal_forces()
    A = oracle.wetting_A(wl.sigma, wl.xi, wl.theta_eq_deg, wl.pi_n, wl.pi_m)
    base = oracle.nodal_forces(q, wl.faces, sigma=wl.sigma, wetting=True, A=A, xi=wl.xi,
                               n=wl.pi_n, m=wl.pi_m)
    ref = oracle.elastic_reference(wl.nodes, wl.faces)
    _, fe = oracle.elastic_forces(q, ref, wl.faces, Gs=ELASTIC["shear_modulus"],
                                  C=ELASTIC["skalak_c"])
    want = base["phi"] + fe
    assert np.max(np.abs(fe)) > 1e-3 * np.max(np.abs(base["phi"]))  # elasticity matters
    assert np.max(np.abs(pg - want)) <= 1e-13 * np.max(np.abs(want))
    g.close()


@pytest.mark.parametrize("which,steps", [("2d", 150), ("3d", 25)])
def test_full_step_fp64(which, steps):
    wl = small_2d() if which == "2d" else small_3d()
    o, g = pair(wl, iblb.FP64)
    assert o.step(steps) == 0
    g.step(steps)
    ro, uo, qo = o.fields()
    rg, ug, qg = g.fields()
    m = fluid_mask(o.shape, wl.dim)
    assert rel_l2(rg[m] - 1.0, ro[m] - 1.0) < 1e-10
    assert rel_l2(ug[:, m], uo[: wl.dim, m]) < 1e-10
    assert np.max(np.abs(qg - qo)) < 1e-11
    # the elastic run differs from the clean drop
    c = oracle_from_workload(wl)
    c.set_equilibrium(shear_field(o.shape, wl.dim, 2e-3))
    c.step(steps)
    assert np.max(np.abs(c.fields()[2] - qo)) > 1e-6
    g.close()


@pytest.mark.parametrize("which,steps", [("2d", 150), ("3d", 25)])
def test_full_step_fp32(which, steps):
    wl = small_2d() if which == "2d" else small_3d()
    o, g = pair(wl, iblb.FP32_DEV)
    assert o.step(steps) == 0
    g.step(steps)
    ro, uo, qo = o.fields()
    rg, ug, qg = g.fields()
    m = fluid_mask(o.shape, wl.dim)
    assert rel_l2(ug[:, m], uo[: wl.dim, m]) < 1e-5
    assert rel_l2(rg[m] - 1.0, ro[m] - 1.0) < 1e-5
    g.close()


def test_batch_elastic_slot_matches_single_engine():
    wl = small_2d(nx=64, ny=30)
    steps = 200
    b = iblb.Batch(iblb.D2Q9, iblb.FP64, 1 * GB, max_slots=4)
    s = b.admit_workload(wl, n_steps=steps, **ELASTIC)
    b.admit_workload(small_2d(nx=48, ny=28, R=5.0), n_steps=steps + 10)
    b.run(steps)
    rb, ub, qb = b.fields(s)
    g = iblb.Simulation.from_workload(wl, **ELASTIC)
    g.step(steps)
    rg, ug, qg = g.fields()
    m = fluid_mask(rg.shape, 2)
    assert rel_l2(ub[:, m], ug[:, m]) < 1e-12
    assert np.max(np.abs(qb - qg)) < 1e-12
    # and against the oracle
    o = oracle_from_workload(wl, **ELASTIC)
    assert o.step(steps) == 0
    assert np.max(np.abs(qb - o.fields()[2])) < 1e-11
    g.close()
    b.close()


def test_rejects_bad_elastic_parameters():
    with pytest.raises(iblb.IBLBError):
        iblb.Simulation(iblb.D2Q9, 32, 24, shear_modulus=-1.0)
    with pytest.raises(iblb.IBLBError):
        iblb.Simulation(iblb.D2Q9, 32, 24, shear_modulus=1e-3, skalak_c=-0.6)
