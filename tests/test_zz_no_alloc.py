"""iblb_mass_static: the mass reduction for callers that cannot allocate
device memory when they need it (for example a process that reserved all of
its GPU memory up front).  Its partial sums live in a static device array
inside the library; the test checks it, through the C-ABI, against the mass
that iblb_observables reports for the same populations and against a host
FP64 sum of the array it uploads, on two calls in a row; it checks that a
second call leaves the device's free memory unchanged, and that a lattice
beyond the static array is refused."""
import math

import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import iblb
from paper_2604_17463_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    (9, (64, 40, 1), True, iblb.FP32_DEV),
    (19, (32, 24, 20), True, iblb.FP32_DEV),
    (19, (24, 16, 12), False, iblb.FP64),
    (9, (40, 30, 1), True, iblb.FP16_DEV),
    (19, (256, 64, 40), True, iblb.FP32_DEV),   # several partials per call
]


def storage_form(f, w, storage):
    """The library's storage form of populations f: deviations f - w, as
    double, float, or binary16 scaled by 2^16 (float first, as the library)."""
    dev = f.reshape(f.shape[0], -1) - w[:, None]
    if storage == iblb.FP64:
        return dev
    if storage == iblb.FP32_DEV:
        return dev.astype(np.float32)
    return (dev.astype(np.float32) * np.float32(65536.0)).astype(np.float16)


def host_mass(stored, Q, dims, walls, storage):
    """FP64 sum over the fluid cells of 1 + sum_i (f_i - w_i), taken from the
    stored form itself (binary16 divided by its scale 2^16)."""
    nx, ny, nz = dims
    dev = np.asarray(stored, dtype=np.float64).reshape(Q, nz, ny, nx)
    if storage == iblb.FP16_DEV:
        dev = dev / 65536.0
    cell = 1.0 + dev.sum(axis=0)
    if walls:
        if Q == 9:
            cell = cell[:, 1:ny - 1, :]
        else:
            cell = cell[1:nz - 1]
    return float(cell.sum())


@pytest.mark.parametrize("Q,dims,walls,storage", CASES)
def test_mass_static_matches_observables(Q, dims, walls, storage):
    import torch
    nx, ny, nz = dims
    _, w, _ = oracle.lattice(Q)
    shape = (Q, nz, ny, nx)
    f = w.reshape(Q, 1, 1, 1) * (1.0 + W.random_perturbation(shape, seed=nx + ny + nz, scale=0.05))
    sim = iblb.Simulation(Q, nx, ny, nz, tau=0.9, walls=walls, wetting=False, storage=storage)
    sim.set_populations(f)
    ref = sim.observables()["mass"]
    sim.close()

    stored = np.ascontiguousarray(storage_form(f, w, storage))
    href = host_mass(stored, Q, dims, walls, storage)
    f_dev = torch.from_numpy(stored).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        iblb.iblb_mass_static(f_dev.data_ptr(), Q, storage, nx, ny, nz, int(walls), 0,
                              out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert math.isclose(out.item(), ref, rel_tol=1e-12), (out.item(), ref)
        assert math.isclose(out.item(), href, rel_tol=1e-12), (out.item(), href)


def test_mass_static_two_sizes_in_a_row():
    # a large call then a small one: the small call must not pick up the
    # partials the large call left in the shared array
    import torch
    results = []
    for dims in ((256, 64, 40), (16, 12, 10)):
        nx, ny, nz = dims
        _, w, _ = oracle.lattice(19)
        f = w.reshape(19, 1, 1, 1) * (1.0 + W.random_perturbation((19, nz, ny, nx), seed=3, scale=0.02))
        sim = iblb.Simulation(19, nx, ny, nz, tau=0.9, walls=True, wetting=False,
                              storage=iblb.FP32_DEV)
        sim.set_populations(f)
        ref = sim.observables()["mass"]
        sim.close()
        f_dev = torch.from_numpy(storage_form(f, w, iblb.FP32_DEV)).cuda()
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        iblb.iblb_mass_static(f_dev.data_ptr(), 19, iblb.FP32_DEV, nx, ny, nz, 1, 0,
                              out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        results.append((out.item(), ref))
    for got, ref in results:
        assert math.isclose(got, ref, rel_tol=1e-12)


def test_mass_static_allocates_no_device_memory():
    # after a first call (which does the per-device set-up), further calls
    # leave the device's free memory exactly as it was
    import torch
    nx, ny, nz = 96, 64, 48
    _, w, _ = oracle.lattice(19)
    f = w.reshape(19, 1, 1, 1) * (1.0 + W.random_perturbation((19, nz, ny, nx), seed=11, scale=0.02))
    stored = np.ascontiguousarray(storage_form(f, w, iblb.FP32_DEV))
    href = host_mass(stored, 19, (nx, ny, nz), True, iblb.FP32_DEV)
    f_dev = torch.from_numpy(stored).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    iblb.iblb_mass_static(f_dev.data_ptr(), 19, iblb.FP32_DEV, nx, ny, nz, 1, 0, out.data_ptr(), stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        iblb.iblb_mass_static(f_dev.data_ptr(), 19, iblb.FP32_DEV, nx, ny, nz, 1, 0,
                              out.data_ptr(), stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert math.isclose(out.item(), href, rel_tol=1e-12)


def test_mass_static_rejects_lattice_beyond_scratch():
    import torch
    tiny = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 1100^3 cells need more partials than the static array holds; refused
    # before any kernel is launched
    with pytest.raises(iblb.IBLBError) as e:
        iblb.iblb_mass_static(tiny.data_ptr(), 19, iblb.FP32_DEV, 1100, 1100, 1100, 1, 0,
                              out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 1
