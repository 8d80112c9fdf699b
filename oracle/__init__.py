"""Plain FP64 CPU oracle of the IBLB wetting time step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never imports, links or calls it, and the
two share no code: the C source here (``iblb_oracle.c``) follows Sec. 2 of the
paper (Eq. 1-11) written out step by step in FP64.

The shared library is compiled in-tree with gcc (``-O2 -ffp-contract=off``)
under ``oracle/_build`` on first use or by :func:`build`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iblb_oracle.c")
_HDR = os.path.join(_HERE, "iblb_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

D2Q9 = 9
D3Q19 = 19


class Params(ctypes.Structure):
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
        ("tau_out", ctypes.c_double),
        ("wall_u_lo", ctypes.c_double * 3),
        ("wall_u_hi", ctypes.c_double * 3),
        ("shear_modulus", ctypes.c_double),
        ("skalak_c", ctypes.c_double),
    ]


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
        return {
            "mass": self.mass,
            "volume": self.volume,
            "height": self.height,
            "theta_deg": self.theta_deg,
            "r_cl": self.r_cl,
            "film": self.film,
            "d_min": self.d_min,
            "centre": list(self.centre),
            "radius": self.radius,
        }


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP64, no FMA contraction)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


_OMP_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_omp.so")
_omp_lib = None


def build_openmp(force: bool = False) -> str:
    """The same oracle source compiled with -fopenmp: its stream-collide rows
    run on all host cores with unchanged arithmetic per cell.  Used only to
    time the oracle across the host's cores."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_OMP_LIB_PATH) and os.path.getmtime(_OMP_LIB_PATH) >= newest:
            return _OMP_LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _OMP_LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OMP_LIB_PATH)
        return _OMP_LIB_PATH


def _load_openmp():
    global _omp_lib
    if _omp_lib is None:
        _omp_lib = _bind(ctypes.CDLL(build_openmp()))
    return _omp_lib


def _load():
    global _lib
    if _lib is not None:
        return _lib
    _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    vp = ctypes.c_void_p
    lib.or_lattice.argtypes = [ctypes.c_int, ip, dp, ip]
    lib.or_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
    lib.or_guo_source.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp]
    lib.or_delta4.argtypes = [ctypes.c_double]
    lib.or_delta4.restype = ctypes.c_double
    lib.or_wetting_A.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int]
    lib.or_wetting_A.restype = ctypes.c_double
    lib.or_wetting_Pi.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double]
    lib.or_wetting_Pi.restype = ctypes.c_double
    lib.or_nodal_forces.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, dp, dp, dp, dp, dp]
    lib.or_sim_create.argtypes = [ctypes.POINTER(Params)]
    lib.or_sim_create.restype = vp
    lib.or_sim_destroy.argtypes = [vp]
    lib.or_sim_set_interface.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int, ip]
    lib.or_sim_set_populations.argtypes = [vp, dp]
    lib.or_sim_get_populations.argtypes = [vp, dp]
    lib.or_sim_step.argtypes = [vp, ctypes.c_int]
    lib.or_sim_get_fields.argtypes = [vp, dp, dp, dp]
    lib.or_sim_force_field.argtypes = [vp, dp]
    lib.or_sim_interpolate.argtypes = [vp, dp, dp]
    lib.or_sim_spread.argtypes = [vp, dp, dp]
    lib.or_sim_nodal_forces.argtypes = [vp, dp, dp, dp]
    lib.or_sim_observables.argtypes = [vp, ctypes.POINTER(Obs)]
    lib.or_sim_inside_mask.argtypes = [vp, ctypes.POINTER(ctypes.c_ubyte)]
    lib.or_sim_set_equilibrium.argtypes = [vp, dp, dp]
    lib.or_deformation.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip, dp]
    lib.or_skalak_W.argtypes = [ctypes.c_double] * 4
    lib.or_skalak_W.restype = ctypes.c_double
    lib.or_elastic_reference.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip, dp]
    lib.or_elastic_forces.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip, dp,
                                      ctypes.c_double, ctypes.c_double, dp]
    lib.or_elastic_forces.restype = ctypes.c_double
    lib.or_sim_A.argtypes = [vp]
    lib.or_sim_A.restype = ctypes.c_double
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if a is not None else None


# ---------------------------------------------------------------- pointwise
def lattice(Q: int):
    """(c [Q,3] int, w [Q], opp [Q]) of the D2Q9 / D3Q19 stencil."""
    lib = _load()
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    if lib.or_lattice(Q, _iptr(c), _dptr(w), _iptr(opp)) != 0:
        raise ValueError(f"unsupported lattice Q={Q}")
    return c, w, opp


def equilibrium(Q: int, rho: float, u) -> np.ndarray:
    u3 = np.zeros(3)
    u3[: len(u)] = u
    out = np.zeros(Q)
    _load().or_equilibrium(Q, float(rho), _dptr(u3), _dptr(out))
    return out


def guo_source(Q: int, tau: float, u, F) -> np.ndarray:
    u3 = np.zeros(3)
    u3[: len(u)] = u
    F3 = np.zeros(3)
    F3[: len(F)] = F
    out = np.zeros(Q)
    _load().or_guo_source(Q, float(tau), _dptr(u3), _dptr(F3), _dptr(out))
    return out


def delta4(r: float) -> float:
    return _load().or_delta4(float(r))


def wetting_A(sigma, xi, theta_eq_deg, n, m) -> float:
    return _load().or_wetting_A(float(sigma), float(xi), float(theta_eq_deg), int(n), int(m))


def wetting_Pi(A, xi, n, m, d) -> float:
    return _load().or_wetting_Pi(float(A), float(xi), int(n), int(m), float(d))


def nodal_forces(q, tri=None, *, sigma, wetting=False, A=0.0, xi=1.0, n=9, m=3,
                 wall_plane=0.5):
    """Nodal forces of an interface. q [N, dim]; tri [M, 3] for dim = 3.

    Returns dict of phi, phi_sigma, phi_pi, normal ([N, dim]) and chi ([N]),
    plus 'bad' (node at or below the wall plane)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    N, dim = q.shape
    t = None if tri is None else np.ascontiguousarray(tri, dtype=np.int32)
    M = 0 if t is None else t.shape[0]
    out = {k: np.zeros((N, dim)) for k in ("phi", "phi_sigma", "phi_pi", "normal")}
    out["chi"] = np.zeros(N)
    bad = _load().or_nodal_forces(dim, N, _dptr(q), M, _iptr(t), float(sigma), int(bool(wetting)),
                                  float(A), float(xi), int(n), int(m), float(wall_plane),
                                  _dptr(out["phi"]), _dptr(out["phi_sigma"]),
                                  _dptr(out["phi_pi"]), _dptr(out["normal"]), _dptr(out["chi"]))
    out["bad"] = bool(bad)
    return out


def skalak_W(Gs, C, I1, I2) -> float:
    """Skalak strain energy per unit reference area from the invariants."""
    return _load().or_skalak_W(float(Gs), float(C), float(I1), float(I2))


def elastic_reference(q0, tri=None) -> np.ndarray:
    """Elastic reference data of an interface at positions q0 (see the C
    header): [M, 5] per face in 3D, [N] reference segment lengths in 2D."""
    q0 = np.ascontiguousarray(q0, dtype=np.float64)
    N, dim = q0.shape
    t = None if tri is None else np.ascontiguousarray(tri, dtype=np.int32)
    M = 0 if t is None else t.shape[0]
    ref = np.zeros(5 * M if dim == 3 else N)
    _load().or_elastic_reference(dim, N, _dptr(q0), M, _iptr(t), _dptr(ref))
    return ref.reshape(M, 5) if dim == 3 else ref


def elastic_forces(q, ref, tri=None, *, Gs, C):
    """(total Skalak energy, nodal forces -dE/dq [N, dim]) at positions q."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    N, dim = q.shape
    t = None if tri is None else np.ascontiguousarray(tri, dtype=np.int32)
    M = 0 if t is None else t.shape[0]
    r = np.ascontiguousarray(ref, dtype=np.float64).ravel()
    f = np.zeros((N, dim))
    E = _load().or_elastic_forces(dim, N, _dptr(q), M, _iptr(t), _dptr(r), float(Gs), float(C),
                                  _dptr(f))
    return E, f


def deformation(q, tri=None) -> dict:
    """Deformation index D = (r1 - r3)/(r1 + r3) of a closed ring (q [N, 2])
    or outward mesh (q [N, 3], tri [M, 3]) in the shear plane (Sec. 4, Eq. 15)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    N, dim = q.shape
    t = None if tri is None else np.ascontiguousarray(tri, dtype=np.int32)
    out = np.zeros(5)
    _load().or_deformation(dim, N, _dptr(q), 0 if t is None else t.shape[0], _iptr(t), _dptr(out))
    return dict(D=out[0], r1=out[1], r3=out[2], angle_deg=out[3], volume=out[4])


# ---------------------------------------------------------------- simulation
class Sim:
    """One oracle simulation. Fields use the layout [component][z][y][x]."""

    def __init__(self, lattice: int, nx: int, ny: int, nz: int = 1, *, tau=1.0, walls=True,
                 wetting=True, sigma=1e-3, xi=1.0, theta_eq_deg=90.0, pi_n=9, pi_m=3,
                 body_force=(0.0, 0.0, 0.0), tau_out=0.0, wall_u_lo=(0.0, 0.0, 0.0),
                 wall_u_hi=(0.0, 0.0, 0.0), shear_modulus=0.0, skalak_c=0.0,
                 openmp=False):
        # openmp: the -fopenmp build (threads from OMP_NUM_THREADS), for timing
        self._lib = _load_openmp() if openmp else _load()
        p = Params()
        p.lattice = lattice
        p.nx, p.ny, p.nz = nx, ny, (1 if lattice == D2Q9 else nz)
        p.walls = int(bool(walls))
        p.wetting = int(bool(wetting))
        p.tau = tau
        p.sigma = sigma
        p.xi = xi
        p.theta_eq_deg = theta_eq_deg
        p.pi_n, p.pi_m = pi_n, pi_m
        for k in range(3):
            p.body_force[k] = body_force[k] if k < len(body_force) else 0.0
        p.tau_out = tau_out
        for k in range(3):
            p.wall_u_lo[k] = wall_u_lo[k] if k < len(wall_u_lo) else 0.0
            p.wall_u_hi[k] = wall_u_hi[k] if k < len(wall_u_hi) else 0.0
        p.shear_modulus = shear_modulus
        p.skalak_c = skalak_c
        self.params = p
        self.Q = lattice
        self.dim = 2 if lattice == D2Q9 else 3
        self.shape = (p.nz, p.ny, p.nx)
        self.ncell = p.nx * p.ny * p.nz
        self._h = self._lib.or_sim_create(ctypes.byref(p))
        if not self._h:
            raise ValueError("oracle: bad parameters")
        self.N = 0
        self.M = 0

    def close(self):
        if self._h:
            self._lib.or_sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def A(self) -> float:
        return self._lib.or_sim_A(self._h)

    def set_interface(self, q, tri=None):
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, self.dim)
        t = None if tri is None else np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        self._tri = t
        self.N = q.shape[0]
        self.M = self.N if self.dim == 2 else (0 if t is None else t.shape[0])
        self._lib.or_sim_set_interface(self._h, self.N, _dptr(q), 0 if t is None else t.shape[0],
                                       _iptr(t))

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.Q, self.ncell)
        self._lib.or_sim_set_populations(self._h, _dptr(f))

    def populations(self) -> np.ndarray:
        f = np.zeros((self.Q, self.ncell))
        self._lib.or_sim_get_populations(self._h, _dptr(f))
        return f.reshape((self.Q,) + self.shape)

    def step(self, n: int = 1) -> int:
        return self._lib.or_sim_step(self._h, int(n))

    def fields(self):
        rho = np.zeros(self.ncell)
        u = np.zeros(3 * self.ncell)
        q = np.zeros(max(self.N, 1) * self.dim)
        self._lib.or_sim_get_fields(self._h, _dptr(rho), _dptr(u), _dptr(q))
        return (rho.reshape(self.shape), u.reshape((3,) + self.shape),
                q[: self.N * self.dim].reshape(self.N, self.dim))

    def force_field(self):
        F = np.zeros(3 * self.ncell)
        bad = self._lib.or_sim_force_field(self._h, _dptr(F))
        return F.reshape((3,) + self.shape), bool(bad)

    def interpolate(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(3 * self.ncell)
        qd = np.zeros(max(self.N, 1) * self.dim)
        self._lib.or_sim_interpolate(self._h, _dptr(u), _dptr(qd))
        return qd[: self.N * self.dim].reshape(self.N, self.dim)

    def spread(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(self.N * self.dim)
        F = np.zeros(3 * self.ncell)
        self._lib.or_sim_spread(self._h, _dptr(phi), _dptr(F))
        return F.reshape((3,) + self.shape)

    def nodal_forces(self):
        phi = np.zeros(max(self.N, 1) * self.dim)
        nrm = np.zeros(max(self.N, 1) * self.dim)
        chi = np.zeros(max(self.N, 1))
        bad = self._lib.or_sim_nodal_forces(self._h, _dptr(phi), _dptr(nrm), _dptr(chi))
        n = self.N * self.dim
        return (phi[:n].reshape(self.N, self.dim), nrm[:n].reshape(self.N, self.dim),
                chi[: self.N], bool(bad))

    def set_equilibrium(self, u, rho=None):
        """f = f_eq(rho, u) (Eq. 3); u [dim] + lattice shape, rho lattice shape or None (1)."""
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.dim, self.ncell)
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ncell)
        self._lib.or_sim_set_equilibrium(self._h, None if r is None else _dptr(r), _dptr(u))

    def deformation(self) -> dict:
        """Deformation index of the current interface (Sec. 4, Eq. 15)."""
        return deformation(self.fields()[2], getattr(self, "_tri", None))

    def inside_mask(self) -> np.ndarray:
        m = np.zeros(self.ncell, dtype=np.uint8)
        self._lib.or_sim_inside_mask(self._h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        return m.reshape(self.shape)

    def observables(self) -> dict:
        o = Obs()
        self._lib.or_sim_observables(self._h, ctypes.byref(o))
        return o.as_dict()
