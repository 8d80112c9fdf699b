"""Host-side logic of the C-ABI that needs no GPU.

- iblb_create refuses bad configurations before any device call.
- iblb_batch_create refuses bad arguments the same way.
- iblb_batch_footprint is pure host arithmetic, so its sizes can be checked
  against the buffers a slot must hold: two population buffers, the
  moments, the force density, the band flags and the interface arrays.

Every call here returns before CUDA is touched: the library is only loaded.
"""
import ctypes
import math

import pytest

from paper_2604_17463_gb300 import iblb

EINVAL = 1


def lib():
    return iblb.load()


def create_status(**kw):
    lattice = kw.pop("lattice", iblb.D2Q9)
    nx, ny, nz = kw.pop("nx", 40), kw.pop("ny", 30), kw.pop("nz", 20)
    cfg = iblb.make_config(lattice, nx, ny, nz, **kw)
    h = ctypes.c_void_p(12345)
    st = lib().iblb_create(ctypes.byref(cfg), None, ctypes.byref(h))
    return st, h.value


def raw_status(cfg):
    h = ctypes.c_void_p(12345)
    st = lib().iblb_create(ctypes.byref(cfg), None, ctypes.byref(h))
    return st, h.value


BAD = {
    "zero width": dict(nx=0),
    "negative height": dict(ny=-3),
    "walls need three layers (2D)": dict(ny=2),
    "walls need three layers (3D)": dict(lattice=iblb.D3Q19, nz=2),
    "tau at the stability limit": dict(tau=0.5),
    "tau below it": dict(tau=0.3),
    "tau not finite": dict(tau=math.nan),
    "storage out of range": dict(storage=5),
    "wetting without walls": dict(walls=False),
    "wetting with xi = 0": dict(xi=0.0),
    "wetting with n <= m": dict(pi_n=3, pi_m=3),
    "wetting with m < 2": dict(pi_n=9, pi_m=1),
    "binary16 scale exponent above 24": dict(fp16_scale_exp=25),
    "negative binary16 scale exponent": dict(fp16_scale_exp=-1),
    "2D height above 65535": dict(ny=70000),
    "3D depth above 65535": dict(lattice=iblb.D3Q19, nz=70000, nx=4, ny=4),
    "2^32 cells": dict(lattice=iblb.D3Q19, nx=65536, ny=65536, nz=1, walls=False, wetting=False),
    "outer tau at the limit": dict(tau_out=0.5),
    "outer tau not finite": dict(tau_out=math.inf),
    "negative shear modulus": dict(shear_modulus=-1e-3),
    "area-dilation modulus at -1/2": dict(shear_modulus=1e-3, skalak_c=-0.5),
    "wall speed above 0.3": dict(wall_u_hi=(0.31, 0.0, 0.0)),
    "wall speed not finite": dict(wall_u_lo=(math.nan, 0.0, 0.0)),
    "wall velocity normal to the wall (2D)": dict(wall_u_hi=(0.0, 0.01, 0.0)),
    "out-of-plane wall velocity (2D)": dict(wall_u_hi=(0.0, 0.0, 0.01)),
    "wall velocity normal to the wall (3D)": dict(lattice=iblb.D3Q19, wall_u_lo=(0.0, 0.0, 0.01)),
    "moving walls without walls": dict(walls=False, wetting=False, wall_u_hi=(0.01, 0.0, 0.0)),
}


@pytest.mark.parametrize("why", list(BAD))
def test_create_refuses_bad_config(why):
    st, h = create_status(**BAD[why])
    assert st == EINVAL, why
    assert h is None  # *out is cleared
    lib().iblb_last_error.restype = ctypes.c_char_p
    lib().iblb_last_error.argtypes = [ctypes.c_void_p]
    assert b"invalid configuration" in lib().iblb_last_error(None)


def test_create_refuses_bad_lattice_and_null_arguments():
    cfg = iblb.make_config(iblb.D2Q9, 40, 30)
    cfg.lattice = 7
    assert raw_status(cfg) == (EINVAL, None)
    h = ctypes.c_void_p()
    assert lib().iblb_create(None, None, ctypes.byref(h)) == EINVAL
    cfg = iblb.make_config(iblb.D2Q9, 40, 30)
    assert lib().iblb_create(ctypes.byref(cfg), None, None) == EINVAL


@pytest.mark.parametrize("lattice,storage,budget,max_slots", [
    (7, iblb.FP32_DEV, 1 << 30, 4),
    (iblb.D2Q9, 3, 1 << 30, 4),
    (iblb.D2Q9, -1, 1 << 30, 4),
    (iblb.D3Q19, iblb.FP32_DEV, 1 << 30, 0),
    (iblb.D3Q19, iblb.FP32_DEV, 1 << 30, (1 << 20) + 1),
    (iblb.D2Q9, iblb.FP64, 16, 4),
])
def test_batch_create_refuses_bad_arguments(lattice, storage, budget, max_slots):
    b = ctypes.c_void_p(12345)
    st = lib().iblb_batch_create(lattice, storage, budget, max_slots, None, ctypes.byref(b))
    assert st == EINVAL
    assert b.value is None


def footprint(lattice, nx, ny, nz=1, nodes=0, faces=0, **kw):
    cfg = iblb.make_config(lattice, nx, ny, nz, **kw)
    return lib().iblb_batch_footprint(ctypes.byref(cfg), nodes, faces)


ELT = {iblb.FP64: 8, iblb.FP32_DEV: 4, iblb.FP16_DEV: 2}


@pytest.mark.parametrize("storage", [iblb.FP64, iblb.FP32_DEV, iblb.FP16_DEV])
@pytest.mark.parametrize("lattice,dims", [(iblb.D2Q9, (97, 31, 1)), (iblb.D3Q19, (33, 29, 21))])
def test_footprint_holds_every_buffer(storage, lattice, dims):
    nx, ny, nz = dims
    dim = 2 if lattice == iblb.D2Q9 else 3
    ncell = nx * ny * nz
    relt = 8 if storage == iblb.FP64 else 4
    pops = 2 * lattice * ncell * ELT[storage]          # two population buffers
    moments = (1 + dim) * ncell * relt                  # density and velocity
    force = dim * ncell * relt                          # force density
    fp = footprint(lattice, nx, ny, nz, storage=storage)
    assert fp >= pops + moments + force
    # and nothing of the order of a third population buffer on top
    assert fp < pops + moments + force + lattice * ncell * ELT[storage] // 2 + (1 << 16)
    # interface arrays: FP64 positions and nodal forces at least (each array
    # starts on a 256-byte boundary and an empty one still takes a block)
    n, m = 500, (996 if dim == 3 else 0)
    fpi = footprint(lattice, nx, ny, nz, nodes=n, faces=m, storage=storage)
    assert fpi - fp >= 2 * n * dim * 8 + (m * 3 * 4 if dim == 3 else 0) - 8 * 256


def test_footprint_orders_and_extras():
    args = (iblb.D3Q19, 40, 36, 28)
    f64, f32, f16 = (footprint(*args, nodes=642, faces=1280, storage=s)
                     for s in (iblb.FP64, iblb.FP32_DEV, iblb.FP16_DEV))
    assert f64 > f32 > f16
    base = footprint(*args, nodes=642, faces=1280, storage=iblb.FP32_DEV)
    # viscosity ratio: a crossing table per lattice column
    assert footprint(*args, nodes=642, faces=1280, storage=iblb.FP32_DEV, tau_out=2.0) > base
    # tau_out equal to tau is no ratio
    assert footprint(*args, nodes=642, faces=1280, storage=iblb.FP32_DEV, tau_out=1.0) == base
    # elastic interface: reference-shape data per face
    assert footprint(*args, nodes=642, faces=1280, storage=iblb.FP32_DEV, shear_modulus=1e-3) > base
    assert lib().iblb_batch_footprint(None, 10, 0) == 0
