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
    (9, (46, 9, 1), True),        # pairs: row ends inside the first warp
    (9, (100, 8, 1), False),      # pairs: row ends inside the second warp
    (9, (45, 9, 1), True),        # odd width: only the plain kernel applies
    (19, (256, 5, 6), True),      # D3Q19, fewer tiles than CTAs
    (19, (64, 7, 5), True),       # D3Q19, y seam inside a tile
    (19, (2048, 3, 4), False),    # D3Q19 segment mode, periodic
    (19, (70, 6, 5), True),       # D3Q19 pairs, ragged warp
]


def applies(variant, Q, nx, storage):
    """Whether a stream-collide variant can run on this shape (else the
    library falls back to the plain kernel)."""
    if variant == 2:
        return storage != iblb.FP64 and nx % 2 == 0
    if variant == 3:
        return storage != iblb.FP64 and Q == 19
    return variant == 0


@pytest.mark.parametrize("Q,dims,walls", CASES)
@pytest.mark.parametrize("storage", [iblb.FP64, iblb.FP32_DEV, iblb.FP16_DEV])
def test_kernel_variants_match_plain_and_oracle(Q, dims, walls, storage):
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    body = (2e-6, -1e-6, 5e-7 if Q == 19 else 0.0)
    f0 = near_eq(Q, shape, seed=nx + ny)
    out = {}
    for variant in (0, 1, 2, 3):
        g = iblb.Simulation(Q, nx, ny, nz, tau=0.83, walls=walls, wetting=False, body_force=body,
                            storage=storage)
        g.set_tuning(variant, rows_per_tile=3)
        if variant in (2, 3):
            assert g.variant == (variant if applies(variant, Q, nx, storage) else 0)
        g.set_populations(f0)
        g.step(4)
        out[variant] = g.populations()
        g.close()
    m = fluid_mask(shape, 2 if Q == 9 else 3, walls)
    # same arithmetic up to FMA placement: agreement to the storage format's
    # last bits; binary16 stores round stochastically with random bits that
    # differ between kernels, so up to one unit in the last place there
    # (populations here have |g| < 1/32, i.e. below 2048 once scaled by 2^16,
    # where the binary16 spacing is at most 1: one ulp <= 2^-16 unscaled)
    tol = {iblb.FP64: 1e-15, iblb.FP32_DEV: 2e-7, iblb.FP16_DEV: 2.0 ** -16 * 1.01}[storage]
    for variant in (1, 2, 3):
        assert np.max(np.abs(out[variant][:, m] - out[0][:, m])) < tol, variant
    if storage == iblb.FP64:
        o = oracle.Sim(Q, nx, ny, nz, tau=0.83, walls=walls, wetting=False, body_force=body)
        o.set_populations(f0)
        o.step(4)
        assert np.max(np.abs(out[0][:, m] - o.populations()[:, m])) < 1e-14


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("storage,tol", [(iblb.FP64, 1e-10), (iblb.FP32_DEV, 1e-5)])
def test_pipeline_full_step_3d_drop(storage, tol, variant):
    # a drop on a lattice whose width selects the pipelined kernel
    R, xi = 6.0, 1.0
    nodes, faces = W.icosphere(2, R, (128.3, 9.7, W.WALL_PLANE + R + 2 * xi))
    wl = W.Workload("pipe3d", 19, 256, 20, 18, 0.8, 5e-3, xi, 75.0, 9, 3, 10, nodes, faces)
    o = oracle_from_workload(wl)
    g = iblb.Simulation.from_workload(wl, storage=storage)
    g.set_tuning(variant)
    assert g.variant == (variant if (variant == 1 or storage != iblb.FP64) else 0)
    o.step(8)
    g.step(8)
    ro, uo, qo = o.fields()
    rg, ug, qg = g.fields()
    m = fluid_mask(o.shape, 3)
    assert rel_l2(ug[:, m], uo[:, m]) < tol
    assert rel_l2(rg[m], ro[m]) < tol
    g.close()


def test_pipeline_used_by_default_on_benchmark_shape():
    wl = W.drop_3d_256x256x128()
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
    assert pick["variant"] in (0, 1, 2, 3)
    a.step(5)
    b.step(5)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fa - fb)) < 1e-7
    _, _, qa = a.fields()
    _, _, qb = b.fields()
    assert np.max(np.abs(qa - qb)) < 1e-9
    a.close()
    b.close()


def test_wait_limit_latches_timeout_and_the_handle_recovers():
    # The pipelined kernel's waits on its shared-memory pipeline are bounded.
    # With a limit of 200 clock cycles (shorter than any bulk copy takes) the
    # consumers give up at their first wait: the launch latches IBLB_ETIMEOUT,
    # which the next synchronising call reports, and the producer still waits
    # for its copies before it exits.  After iblb_clear_faults, with the
    # default limit and the populations set again, the same handle gives
    # exactly the results of a fresh one.
    Q, nx, ny = 9, 256, 64
    f0 = near_eq(Q, (1, ny, nx), seed=77)
    kw = dict(tau=0.8, walls=True, wetting=False, storage=iblb.FP32_DEV)
    g = iblb.Simulation(Q, nx, ny, **kw)
    g.set_populations(f0)
    g.set_tuning(1, rows_per_tile=2, ctas_per_sm=2, consumer_warps=8, wait_limit_cycles=200)
    assert g.variant == 1
    assert g.tuning()["wait_limit_cycles"] == 200
    g.step(3)
    with pytest.raises(iblb.IBLBError) as e:
        g.sync()
    assert e.value.status == 6   # IBLB_ETIMEOUT
    g.clear_faults()
    g.sync()
    g.set_tuning(1, rows_per_tile=2, ctas_per_sm=2, consumer_warps=8)
    g.set_populations(f0)
    g.step(5)
    ref = iblb.Simulation(Q, nx, ny, **kw)
    ref.set_tuning(1, rows_per_tile=2, ctas_per_sm=2, consumer_warps=8)
    ref.set_populations(f0)
    ref.step(5)
    m = fluid_mask((1, ny, nx), 2)   # solid rows are never written
    assert np.array_equal(g.populations()[:, m], ref.populations()[:, m])
    g.close()
    ref.close()
