"""ctypes binding of libiblb (include/iblb.h): argument marshalling only.

Every step of the IBLB time step runs in the CUDA library; this module only
converts numpy arrays and torch streams to the C-ABI's plain pointers.  There
is no CPU fallback: if the library cannot be built or loaded, every call raises.

The functions below carry the names of the C entry points; :class:`Simulation`
is a small convenience wrapper around one handle.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

D2Q9 = 9
D3Q19 = 19
FP64, FP32_DEV, FP16_DEV = 0, 1, 2
STORAGE_NAMES = {"fp64": FP64, "fp32": FP32_DEV, "fp16": FP16_DEV}

IBLB_OK = 0
STATUS = {0: "IBLB_OK", 1: "IBLB_EINVAL", 2: "IBLB_ENOMEM", 3: "IBLB_ECUDA",
          4: "IBLB_ENODE_IN_WALL", 5: "IBLB_ENONFINITE", 6: "IBLB_ETIMEOUT", 7: "IBLB_EAGAIN",
          8: "IBLB_ECLASSIFY"}
K_FORCES, K_SPREAD, K_STREAM_COLLIDE, K_INTERP_ADVECT, K_BAND_CELLS, K_COUNT = 0, 1, 2, 3, 4, 5
KERNEL_NAMES = ["forces", "spread", "stream_collide", "interp_advect", "band_cells"]


class IBLBError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("walls", ctypes.c_int),
        ("wetting", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("xi", ctypes.c_double),
        ("theta_eq_deg", ctypes.c_double),
        ("pi_n", ctypes.c_int),
        ("pi_m", ctypes.c_int),
        ("body_force", ctypes.c_double * 3),
        ("storage", ctypes.c_int),
        ("fp16_scale_exp", ctypes.c_int),
        ("tau_out", ctypes.c_double),
        ("wall_u_lo", ctypes.c_double * 3),
        ("wall_u_hi", ctypes.c_double * 3),
        ("deterministic_spread", ctypes.c_int),
        ("shear_modulus", ctypes.c_double),
        ("skalak_c", ctypes.c_double),
    ]


class Tuning(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int),
        ("block_x", ctypes.c_int),
        ("streaming_stores", ctypes.c_int),
        ("rows_per_tile", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("consumer_warps", ctypes.c_int),
        ("wait_limit_cycles", ctypes.c_longlong),
        ("ib_grouped", ctypes.c_int),
        ("step_overlap", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Obs(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double),
        ("volume", ctypes.c_double),
        ("height", ctypes.c_double),
        ("theta_deg", ctypes.c_double),
        ("r_cl", ctypes.c_double),
        ("film", ctypes.c_double),
        ("d_min", ctypes.c_double),
        ("centre", ctypes.c_double * 3),
        ("radius", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k == "centre" else getattr(self, k))
                for k, _ in self._fields_}


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("slots_used", ctypes.c_int),
        ("slots_active", ctypes.c_int),
        ("slots_done", ctypes.c_int),
        ("arena_bytes", ctypes.c_size_t),
        ("free_bytes", ctypes.c_size_t),
        ("kernel_launches", ctypes.c_longlong),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Build (if stale) and load libiblb.so; raises if that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    st = ctypes.c_int
    sig = {
        "iblb_create": (st, [ctypes.POINTER(Config), vp, ctypes.POINTER(vp)]),
        "iblb_destroy": (None, [vp]),
        "iblb_last_error": (ctypes.c_char_p, [vp]),
        "iblb_status_string": (ctypes.c_char_p, [ip]),
        "iblb_set_interface": (st, [vp, dp, ip, ctypes.POINTER(ctypes.c_int), ip]),
        "iblb_step": (st, [vp, ip]),
        "iblb_sync": (st, [vp]),
        "iblb_clear_faults": (st, [vp]),
        "iblb_read_fields": (st, [vp, dp, dp, dp]),
        "iblb_set_populations": (st, [vp, dp]),
        "iblb_get_populations": (st, [vp, dp]),
        "iblb_observables": (st, [vp, ctypes.POINTER(Obs)]),
        "iblb_nodal_forces": (st, [vp, dp, dp, dp]),
        "iblb_force_field": (st, [vp, dp]),
        "iblb_interpolate": (st, [vp, dp, dp]),
        "iblb_inside_mask": (st, [vp, ctypes.POINTER(ctypes.c_ubyte)]),
        "iblb_set_equilibrium": (st, [vp, dp, dp]),
        "iblb_deformation": (st, [vp, dp]),
        "iblb_step_profiled": (st, [vp, ip, dp]),
        "iblb_set_tuning": (st, [vp, ctypes.POINTER(Tuning)]),
        "iblb_get_tuning": (st, [vp, ctypes.POINTER(Tuning)]),
        "iblb_stream_collide_variant": (ctypes.c_int, [vp]),
        "iblb_autotune": (st, [vp, ip, ctypes.POINTER(Tuning)]),
        "iblb_mass_static": (st, [vp, ip, ip, ip, ip, ip, ip, ip, vp, vp]),
        "iblb_batch_footprint": (ctypes.c_size_t, [ctypes.POINTER(Config), ip, ip]),
        "iblb_batch_create": (st, [ip, ip, ctypes.c_size_t, ip, vp, ctypes.POINTER(vp)]),
        "iblb_batch_destroy": (None, [vp]),
        "iblb_batch_last_error": (ctypes.c_char_p, [vp]),
        "iblb_batch_admit": (st, [vp, ctypes.POINTER(Config), dp, ip, ctypes.POINTER(ctypes.c_int),
                                  ip, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]),
        "iblb_batch_run": (st, [vp, ip, ctypes.POINTER(ctypes.c_int)]),
        "iblb_batch_run_profiled": (st, [vp, ip, ctypes.POINTER(ctypes.c_int), dp, dp]),
        "iblb_batch_sync": (st, [vp]),
        "iblb_batch_poll": (st, [vp, ctypes.POINTER(ctypes.c_int), ip, ctypes.POINTER(ctypes.c_int)]),
        "iblb_batch_slot_status": (st, [vp, ip, ctypes.POINTER(ctypes.c_longlong)]),
        "iblb_batch_observables": (st, [vp, ip, ctypes.POINTER(Obs)]),
        "iblb_batch_read_fields": (st, [vp, ip, dp, dp, dp]),
        "iblb_batch_release": (st, [vp, ip]),
        "iblb_batch_stats": (st, [vp, ctypes.POINTER(BatchInfo)]),
        "iblb_batch_slot_tile": (ctypes.c_int, [vp, ip]),
        "iblb_batch_steps_to_next_completion": (ctypes.c_longlong, [vp]),
        "iblb_stream_bytes_per_step": (ctypes.c_double, [vp]),
        "iblb_fluid_cells": (ctypes.c_longlong, [vp]),
        "iblb_kernel_launch_count": (ctypes.c_longlong, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(h, status: int):
    if status != IBLB_OK:
        lib = load()
        msg = (lib.iblb_last_error(h) or b"").decode()
        raise IBLBError(status, msg)


def current_stream_handle() -> int:
    """The cudaStream_t of torch's current stream (0 if torch has no CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


def make_config(lattice, nx, ny, nz=1, *, tau=1.0, walls=True, wetting=True, sigma=1e-3, xi=1.0,
                theta_eq_deg=90.0, pi_n=9, pi_m=3, body_force=(0.0, 0.0, 0.0), storage=FP64,
                fp16_scale_exp=0, tau_out=0.0, wall_u_lo=(0.0, 0.0, 0.0),
                wall_u_hi=(0.0, 0.0, 0.0), deterministic_spread=False, shear_modulus=0.0,
                skalak_c=0.0) -> Config:
    c = Config()
    c.lattice = lattice
    c.nx, c.ny, c.nz = nx, ny, (1 if lattice == D2Q9 else nz)
    c.walls = int(bool(walls))
    c.wetting = int(bool(wetting))
    c.tau = tau
    c.sigma = sigma
    c.xi = xi
    c.theta_eq_deg = theta_eq_deg
    c.pi_n, c.pi_m = pi_n, pi_m
    for k in range(3):
        c.body_force[k] = body_force[k] if k < len(body_force) else 0.0
    c.storage = STORAGE_NAMES.get(storage, storage) if isinstance(storage, str) else storage
    c.fp16_scale_exp = fp16_scale_exp
    c.tau_out = tau_out
    for k in range(3):
        c.wall_u_lo[k] = wall_u_lo[k] if k < len(wall_u_lo) else 0.0
        c.wall_u_hi[k] = wall_u_hi[k] if k < len(wall_u_hi) else 0.0
    c.deterministic_spread = int(bool(deterministic_spread))
    c.shear_modulus = shear_modulus
    c.skalak_c = skalak_c
    return c


# ------------------------------------------------------------------ C-ABI names
def iblb_create(cfg: Config, stream: Optional[int] = None):
    lib = load()
    h = ctypes.c_void_p()
    s = current_stream_handle() if stream is None else stream
    _check(None, lib.iblb_create(ctypes.byref(cfg), ctypes.c_void_p(s), ctypes.byref(h)))
    return h


def iblb_destroy(h):
    load().iblb_destroy(h)


def iblb_set_interface(h, xyz: np.ndarray, tri: Optional[np.ndarray] = None):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0] if xyz.size else 0
    t = None if tri is None else np.ascontiguousarray(tri, dtype=np.int32)
    tp = None if t is None else t.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    _check(h, load().iblb_set_interface(h, _dptr(xyz) if n else None, n, tp,
                                        0 if t is None else t.shape[0]))


def iblb_step(h, n_steps: int):
    _check(h, load().iblb_step(h, int(n_steps)))


def iblb_sync(h):
    _check(h, load().iblb_sync(h))


def iblb_read_fields(h, rho: Optional[np.ndarray], u: Optional[np.ndarray],
                     xyz: Optional[np.ndarray]):
    _check(h, load().iblb_read_fields(h, _dptr(rho), _dptr(u), _dptr(xyz)))


def iblb_set_populations(h, f: np.ndarray):
    _check(h, load().iblb_set_populations(h, _dptr(np.ascontiguousarray(f, dtype=np.float64))))


def iblb_get_populations(h, f: np.ndarray):
    _check(h, load().iblb_get_populations(h, _dptr(f)))


def iblb_observables(h) -> dict:
    o = Obs()
    _check(h, load().iblb_observables(h, ctypes.byref(o)))
    return o.as_dict()


def iblb_nodal_forces(h, phi, normal, chi):
    _check(h, load().iblb_nodal_forces(h, _dptr(phi), _dptr(normal), _dptr(chi)))


def iblb_force_field(h, F: np.ndarray):
    _check(h, load().iblb_force_field(h, _dptr(F)))


def iblb_interpolate(h, u: np.ndarray, qdot: np.ndarray):
    _check(h, load().iblb_interpolate(h, _dptr(np.ascontiguousarray(u, dtype=np.float64)),
                                      _dptr(qdot)))


def iblb_step_profiled(h, n_steps: int) -> np.ndarray:
    out = np.zeros(K_COUNT)
    _check(h, load().iblb_step_profiled(h, int(n_steps), _dptr(out)))
    return out


def iblb_set_tuning(h, variant: int, block_x: int = 128, streaming_stores: int = 0,
                    rows_per_tile: int = 2, ctas_per_sm: int = 2, consumer_warps: int = 8,
                    wait_limit_cycles: int = 0, ib_grouped: int = 0, step_overlap: int = 0):
    t = Tuning(int(variant), int(block_x), int(streaming_stores), int(rows_per_tile),
               int(ctas_per_sm), int(consumer_warps), int(wait_limit_cycles), int(ib_grouped),
               int(step_overlap))
    _check(h, load().iblb_set_tuning(h, ctypes.byref(t)))


def iblb_get_tuning(h) -> dict:
    t = Tuning()
    _check(h, load().iblb_get_tuning(h, ctypes.byref(t)))
    return t.as_dict()


def iblb_autotune(h, trials: int = 10) -> dict:
    t = Tuning()
    _check(h, load().iblb_autotune(h, int(trials), ctypes.byref(t)))
    return t.as_dict()


def iblb_mass_static(f_dev_ptr: int, lattice: int, storage: int, nx: int, ny: int, nz: int,
                     walls: int, fp16_scale_exp: int, mass_dev_ptr: int, stream: Optional[int] = None):
    """FP64 mass of a caller-owned device population array, with no device
    allocation (see include/iblb.h); pointers are device addresses."""
    s = current_stream_handle() if stream is None else stream
    st = load().iblb_mass_static(ctypes.c_void_p(f_dev_ptr), int(lattice), int(storage), int(nx),
                                 int(ny), int(nz), int(walls), int(fp16_scale_exp),
                                 ctypes.c_void_p(mass_dev_ptr), ctypes.c_void_p(s))
    if st != IBLB_OK:
        raise IBLBError(st, "iblb_mass_static")


def iblb_stream_collide_variant(h) -> int:
    return load().iblb_stream_collide_variant(h)


def iblb_stream_bytes_per_step(h) -> float:
    return load().iblb_stream_bytes_per_step(h)


def iblb_fluid_cells(h) -> int:
    return load().iblb_fluid_cells(h)


def iblb_kernel_launch_count() -> int:
    return load().iblb_kernel_launch_count()


# ------------------------------------------------------------------ wrapper
class Simulation:
    """One device-resident IBLB simulation (a handle of libiblb)."""

    def __init__(self, lattice, nx, ny, nz=1, stream: Optional[int] = None, **kw):
        self.cfg = make_config(lattice, nx, ny, nz, **kw)
        self.Q = lattice
        self.dim = 2 if lattice == D2Q9 else 3
        self.shape = (self.cfg.nz, ny, nx)
        self.ncell = nx * ny * self.cfg.nz
        self.h = iblb_create(self.cfg, stream)
        self.N = 0

    @classmethod
    def from_workload(cls, wl, storage=FP64, stream=None, **over):
        kw = dict(tau=wl.tau, walls=wl.walls, wetting=wl.wetting, sigma=wl.sigma, xi=wl.xi,
                  theta_eq_deg=wl.theta_eq_deg, pi_n=wl.pi_n, pi_m=wl.pi_m, storage=storage)
        kw.update(over)
        s = cls(wl.lattice, wl.nx, wl.ny, wl.nz, stream=stream, **kw)
        s.set_interface(wl.nodes, wl.faces)
        return s

    def close(self):
        if getattr(self, "h", None):
            iblb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_interface(self, xyz, tri=None):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, self.dim)
        iblb_set_interface(self.h, xyz, tri)
        self.N = xyz.shape[0]

    def step(self, n=1):
        iblb_step(self.h, n)

    def sync(self):
        iblb_sync(self.h)

    def fields(self):
        rho = np.zeros(self.ncell)
        u = np.zeros(self.dim * self.ncell)
        q = np.zeros(max(self.N, 1) * self.dim)
        iblb_read_fields(self.h, rho, u, q)
        return (rho.reshape(self.shape), u.reshape((self.dim,) + self.shape),
                q[: self.N * self.dim].reshape(self.N, self.dim))

    def set_populations(self, f):
        iblb_set_populations(self.h, np.asarray(f, dtype=np.float64).reshape(self.Q, -1))

    def populations(self):
        f = np.zeros((self.Q, self.ncell))
        iblb_get_populations(self.h, f)
        return f.reshape((self.Q,) + self.shape)

    def observables(self):
        return iblb_observables(self.h)

    def nodal_forces(self):
        phi = np.zeros((self.N, self.dim))
        nrm = np.zeros((self.N, self.dim))
        chi = np.zeros(self.N)
        iblb_nodal_forces(self.h, phi, nrm, chi)
        return phi, nrm, chi

    def force_field(self):
        F = np.zeros((self.dim,) + self.shape)
        iblb_force_field(self.h, F)
        return F

    def interpolate(self, u):
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64)[: self.dim])
        qd = np.zeros((self.N, self.dim))
        iblb_interpolate(self.h, u, qd)
        return qd

    def set_tuning(self, variant, block_x=128, streaming_stores=0, rows_per_tile=2,
                   ctas_per_sm=2, consumer_warps=8, wait_limit_cycles=0, ib_grouped=0,
                   step_overlap=0):
        iblb_set_tuning(self.h, variant, block_x, streaming_stores, rows_per_tile, ctas_per_sm,
                        consumer_warps, wait_limit_cycles, ib_grouped, step_overlap)

    def clear_faults(self):
        _check(self.h, load().iblb_clear_faults(self.h))

    def tuning(self):
        return iblb_get_tuning(self.h)

    def autotune(self, trials=10):
        return iblb_autotune(self.h, trials)

    @property
    def variant(self):
        return iblb_stream_collide_variant(self.h)

    def set_equilibrium(self, u, rho=None):
        """Populations = f_eq(rho, u) (Eq. 3); u [dim] + lattice shape."""
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.dim, self.ncell)
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ncell)
        _check(self.h, load().iblb_set_equilibrium(self.h, None if r is None else _dptr(r),
                                                    _dptr(u)))

    def deformation(self):
        """Deformation index of the interface in the shear plane (Sec. 4, Eq. 15)."""
        out = np.zeros(5)
        _check(self.h, load().iblb_deformation(self.h, _dptr(out)))
        return dict(D=out[0], r1=out[1], r3=out[2], angle_deg=out[3], volume=out[4])

    def inside_mask(self):
        m = np.zeros(self.ncell, dtype=np.uint8)
        _check(self.h, load().iblb_inside_mask(
            self.h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))))
        return m.reshape(self.shape)

    def step_profiled(self, n):
        return iblb_step_profiled(self.h, n)

    @property
    def fluid_cells(self):
        return iblb_fluid_cells(self.h)

    @property
    def stream_bytes_per_step(self):
        return iblb_stream_bytes_per_step(self.h)


# ------------------------------------------------------------------ batch
class Batch:
    """Many droplet simulations of one lattice type and storage form advanced
    by shared launches (libiblb's batched engine)."""

    def __init__(self, lattice: int, storage: int, hbm_budget_bytes: int, max_slots: int = 1024,
                 stream: Optional[int] = None):
        lib = load()
        self.lattice = lattice
        self.storage = storage
        self.dim = 2 if lattice == D2Q9 else 3
        h = ctypes.c_void_p()
        s = current_stream_handle() if stream is None else stream
        st = lib.iblb_batch_create(int(lattice), int(storage), int(hbm_budget_bytes),
                                   int(max_slots), ctypes.c_void_p(s), ctypes.byref(h))
        if st != IBLB_OK:
            raise IBLBError(st, "iblb_batch_create")
        self.h = h
        self.max_slots = max_slots
        self.meta = {}

    def _check(self, st):
        if st != IBLB_OK:
            raise IBLBError(st, (load().iblb_batch_last_error(self.h) or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            load().iblb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def footprint(cfg: Config, n_nodes: int, n_faces: int = 0) -> int:
        return int(load().iblb_batch_footprint(ctypes.byref(cfg), int(n_nodes), int(n_faces)))

    def admit(self, cfg: Config, xyz, tri=None, n_steps: int = 1000) -> Optional[int]:
        """Slot index, or None if the batch has no room right now."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, self.dim)
        t = None if tri is None else np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        tp = None if t is None else t.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        slot = ctypes.c_int(-1)
        st = load().iblb_batch_admit(self.h, ctypes.byref(cfg), _dptr(xyz), xyz.shape[0], tp,
                                     0 if t is None else t.shape[0], int(n_steps),
                                     ctypes.byref(slot))
        if st == 7:  # IBLB_EAGAIN
            return None
        self._check(st)
        self.meta[slot.value] = (cfg, xyz.shape[0])
        return slot.value

    def admit_workload(self, wl, n_steps=None, **over) -> Optional[int]:
        kw = dict(tau=wl.tau, walls=wl.walls, wetting=wl.wetting, sigma=wl.sigma, xi=wl.xi,
                  theta_eq_deg=wl.theta_eq_deg, pi_n=wl.pi_n, pi_m=wl.pi_m, storage=self.storage)
        kw.update(over)
        cfg = make_config(wl.lattice, wl.nx, wl.ny, wl.nz, **kw)
        return self.admit(cfg, wl.nodes, wl.faces, wl.steps if n_steps is None else n_steps)

    def run(self, max_steps: int) -> int:
        done = ctypes.c_int(0)
        self._check(load().iblb_batch_run(self.h, int(max_steps), ctypes.byref(done)))
        return done.value

    def run_profiled(self, max_steps: int):
        """(completed, per-phase device ms [K_COUNT], stream-collide bytes)."""
        done = ctypes.c_int(0)
        kms = np.zeros(K_COUNT)
        nb = ctypes.c_double(0.0)
        self._check(load().iblb_batch_run_profiled(self.h, int(max_steps), ctypes.byref(done),
                                                   _dptr(kms), ctypes.byref(nb)))
        return done.value, kms, nb.value

    def sync(self):
        self._check(load().iblb_batch_sync(self.h))

    def poll(self):
        n = ctypes.c_int(0)
        buf = (ctypes.c_int * self.max_slots)()
        self._check(load().iblb_batch_poll(self.h, buf, self.max_slots, ctypes.byref(n)))
        return [buf[i] for i in range(min(n.value, self.max_slots))]

    def steps_done(self, slot: int) -> int:
        v = ctypes.c_longlong(0)
        self._check(load().iblb_batch_slot_status(self.h, int(slot), ctypes.byref(v)))
        return v.value

    def observables(self, slot: int) -> dict:
        o = Obs()
        self._check(load().iblb_batch_observables(self.h, int(slot), ctypes.byref(o)))
        return o.as_dict()

    def fields(self, slot: int):
        cfg, n = self.meta[slot]
        nz = 1 if self.dim == 2 else cfg.nz
        ncell = cfg.nx * cfg.ny * nz
        rho = np.zeros(ncell)
        u = np.zeros(self.dim * ncell)
        q = np.zeros(n * self.dim)
        self._check(load().iblb_batch_read_fields(self.h, int(slot), _dptr(rho), _dptr(u),
                                                  _dptr(q)))
        shape = (nz, cfg.ny, cfg.nx)
        return rho.reshape(shape), u.reshape((self.dim,) + shape), q.reshape(n, self.dim)

    def release(self, slot: int):
        self._check(load().iblb_batch_release(self.h, int(slot)))
        self.meta.pop(slot, None)

    def steps_to_next_completion(self) -> int:
        """Steps until the next active slot completes (-1: none active)."""
        return int(load().iblb_batch_steps_to_next_completion(self.h))

    def tile(self, slot: int) -> int:
        return load().iblb_batch_slot_tile(self.h, int(slot))

    def info(self) -> dict:
        i = BatchInfo()
        self._check(load().iblb_batch_stats(self.h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in i._fields_}
