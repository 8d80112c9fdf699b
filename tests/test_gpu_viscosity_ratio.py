"""GPU parity of the viscosity-ratio step (Sec. 2: cells inside the interface
relax with tau, cells outside with tau_out, the two sets found each step by
ray tracing along the lattice columns).

The inside / outside mask is an integer result decided by FP64 crossing
heights and edge-function signs; both sides evaluate the same formulas in
FP64 with every operation rounded on its own, so the masks must agree bit for
bit, ties on shared edges and vertices included.  The full step with
tau_out != tau is compared with the oracle at the single-tau tolerances.
"""
import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import iblb
from paper_2604_17463_gb300 import workloads as W
from helpers import box_mesh, fluid_mask, oracle_from_workload, rel_l2, small_2d, small_3d, star

pytestmark = pytest.mark.gpu


def masks(lattice, dims, nodes, faces=None, walls=False):
    kw = dict(walls=walls, wetting=False, tau=0.8, tau_out=1.1)
    o = oracle.Sim(lattice, *dims, **kw)
    g = iblb.Simulation(lattice, *dims, **kw)
    o.set_interface(nodes, faces)
    g.set_interface(nodes, faces)
    mo, mg = o.inside_mask(), g.inside_mask()
    o.close()
    g.close()
    return mo, mg


@pytest.mark.parametrize("nx,ny,centre", [(48, 40, (23.37, 19.61)), (131, 37, (1.9, 18.2))])
def test_mask_star_polygon_2d(nx, ny, centre):
    # non-convex ring; the second case straddles the periodic seam, ragged width
    mo, mg = masks(9, (nx, ny), star(5, 6.3, 15.1, np.array(centre)))
    assert 0 < mo.sum() < nx * ny
    assert np.array_equal(mg, mo)


def test_mask_ring_through_lattice_points_2d():
    # vertices on integer coordinates: columns through vertices and along
    # vertical edges exercise the half-open tie rule
    sq = np.array([[4, 3], [9, 3], [12, 6], [12, 11], [4, 11], [7, 7]], dtype=np.float64)
    mo, mg = masks(9, (20, 16), sq)
    assert mo.sum() > 0
    assert np.array_equal(mg, mo)


@pytest.mark.parametrize("lo,hi", [((3.3, 2.6, 1.7), (11.2, 9.4, 8.8)), ((3, 2, 2), (11, 9, 8))])
def test_mask_box_3d(lo, hi):
    # the second box has every corner and edge on lattice lines (top-left rule)
    v, tri = box_mesh(lo, hi)
    v = v.astype(np.float64)
    mo, mg = masks(19, (16, 14, 12), v, tri)
    assert mo.sum() > 0
    assert np.array_equal(mg, mo)


@pytest.mark.parametrize("seed,amp", [(0, 0.02), (1, 0.08)])
def test_mask_perturbed_sphere_3d(seed, amp):
    # rough surfaces: the second one crosses some columns 14 times
    q, tri = W.icosphere(4, 7.3, (12.21, 11.87, 10.63))
    rng = np.random.default_rng(seed)
    c = np.array([12.21, 11.87, 10.63])
    r = q - c
    q = c + r * (1.0 + amp * rng.standard_normal((len(q), 1)))
    mo, mg = masks(19, (24, 24, 22), q, tri)
    assert mo.sum() > 0
    assert np.array_equal(mg, mo)


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_mask_of_wall_drop(which):
    wl = small_2d() if which == "2d" else small_3d()
    o = oracle_from_workload(wl, tau_out=1.3)
    g = iblb.Simulation.from_workload(wl, tau_out=1.3)
    assert np.array_equal(g.inside_mask(), o.inside_mask())
    o.step(3)
    g.step(3)
    assert np.array_equal(g.inside_mask(), o.inside_mask())
    o.close()
    g.close()


def test_column_overflow_is_reported():
    # a comb whose teeth cross one column more often than the per-column table holds
    # (20 crossings in the columns 4 <= x <= 13)
    zig = [[14.0 if k % 2 == 0 else 3.5, 2.5 + k] for k in range(20)]
    ring = np.array(zig + [[1.5, 21.5], [1.5, 2.5]], dtype=np.float64)
    g = iblb.Simulation(9, 24, 28, walls=False, wetting=False, tau=0.8, tau_out=1.1)
    g.set_interface(ring)
    with pytest.raises(iblb.IBLBError) as e:
        g.inside_mask()
    assert e.value.status == 8
    g.close()


@pytest.mark.parametrize("which,steps,tau,tau_out", [("2d", 50, 0.9, 0.6), ("2d", 50, 0.7, 1.6),
                                                     ("3d", 12, 0.8, 1.2)])
def test_full_step_two_tau_fp64(which, steps, tau, tau_out):
    wl = small_2d(tau=tau) if which == "2d" else small_3d(tau=tau)
    o = oracle_from_workload(wl, tau_out=tau_out)
    g = iblb.Simulation.from_workload(wl, tau_out=tau_out)
    assert o.step(steps) == 0
    g.step(steps)
    ro, uo, qo = o.fields()
    rg, ug, qg = g.fields()
    m = fluid_mask(o.shape, wl.dim)
    assert rel_l2(rg[m] - 1.0, ro[m] - 1.0) < 1e-10
    assert rel_l2(ug[:, m], uo[: wl.dim, m]) < 1e-10
    assert np.max(np.abs(qg - qo)) < 1e-11
    # the ratio changes the flow: a single-tau run differs
    s = iblb.Simulation.from_workload(wl)
    s.step(steps)
    _, us, _ = s.fields()
    assert rel_l2(us[:, m], uo[: wl.dim, m]) > 1e-4
    s.close()
    g.close()


def test_two_tau_fp32_and_every_tuning():
    wl = small_2d(tau=0.9)
    o = oracle_from_workload(wl, tau_out=0.65)
    assert o.step(200) == 0
    ro, uo, _ = o.fields()
    m = fluid_mask(o.shape, 2)
    for variant in (0, 1, 2):
        g = iblb.Simulation.from_workload(wl, storage=iblb.FP32_DEV, tau_out=0.65)
        g.set_tuning(variant=variant)
        g.step(200)
        rg, ug, _ = g.fields()
        assert rel_l2(rg[m] - 1.0, ro[m] - 1.0) < 1e-5, variant
        assert rel_l2(ug[:, m], uo[:2, m]) < 1e-5, variant
        g.close()


def test_two_tau_launch_count():
    wl = small_2d()
    g = iblb.Simulation.from_workload(wl, tau_out=1.2)
    n0 = iblb.iblb_kernel_launch_count()
    g.step(10)
    g.sync()
    assert iblb.iblb_kernel_launch_count() - n0 == 50
    g.close()


@pytest.mark.parametrize("which", ["2d", "3d"])
@pytest.mark.parametrize("storage,tol", [(iblb.FP64, 1e-12), (iblb.FP32_DEV, 1e-5)])
def test_batch_viscosity_ratio_matches_single_engine(which, storage, tol):
    # a lambda = 4 slot and a lambda = 1 slot in one batch: each equals the
    # single engine, and the lambda = 4 slot differs from the same drop at
    # lambda = 1
    wl = small_2d(nx=48, ny=30) if which == "2d" else small_3d(n=24, nz=20)
    other = small_2d(nx=40, ny=26, R=5.0) if which == "2d" else small_3d(n=20, nz=16, R=4.5)
    steps = 150 if which == "2d" else 40
    tau_out = 0.5 + (wl.tau - 0.5) / 4.0
    b = iblb.Batch(wl.lattice, storage, 1 << 30, max_slots=4)
    s = b.admit_workload(wl, n_steps=steps, tau_out=tau_out)
    r = b.admit_workload(other, n_steps=steps)
    b.run(steps)
    rb, ub, qb = b.fields(s)
    g = iblb.Simulation.from_workload(wl, storage=storage, tau_out=tau_out)
    g.step(steps)
    rg, ug, qg = g.fields()
    m = fluid_mask(rg.shape, wl.dim)
    assert rel_l2(ub[:, m], ug[:, m]) < tol
    assert np.max(np.abs(qb - qg)) < (1e-11 if storage == iblb.FP64 else 1e-4)
    c = iblb.Simulation.from_workload(wl, storage=storage)
    c.step(steps)
    assert np.max(np.abs(c.fields()[2] - qb)) > 1e-6
    rr, ur, qr = b.fields(r)
    g2 = iblb.Simulation.from_workload(other, storage=storage)
    g2.step(steps)
    m2 = fluid_mask(rr.shape, other.dim)
    assert rel_l2(ur[:, m2], g2.fields()[1][:, m2]) < tol
    for x in (g, c, g2):
        x.close()
    b.close()


def test_batch_rejects_bad_tau_out():
    b = iblb.Batch(iblb.D2Q9, iblb.FP32_DEV, 1 << 28, max_slots=4)
    with pytest.raises(iblb.IBLBError):
        b.admit_workload(small_2d(), tau_out=0.4)
    b.close()
