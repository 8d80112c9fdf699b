"""Shared test helpers: building matching oracle / CUDA simulations and
comparing their fields.  Inputs come from the seeded generators only."""
import math

import numpy as np

import oracle
from paper_2604_17463_gb300 import workloads as W


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    num = np.linalg.norm((a - b).ravel())
    return num / den if den > 0 else num


def oracle_from_workload(wl, **over):
    kw = dict(tau=wl.tau, walls=wl.walls, wetting=wl.wetting, sigma=wl.sigma, xi=wl.xi,
              theta_eq_deg=wl.theta_eq_deg, pi_n=wl.pi_n, pi_m=wl.pi_m)
    kw.update(over)
    s = oracle.Sim(wl.lattice, wl.nx, wl.ny, wl.nz, **kw)
    s.set_interface(wl.nodes, wl.faces)
    return s


def fluid_mask(shape, dim, walls=True):
    nz, ny, nx = shape
    m = np.ones(shape, dtype=bool)
    if walls:
        if dim == 2:
            m[:, 0, :] = False
            m[:, ny - 1, :] = False
        else:
            m[0] = False
            m[nz - 1] = False
    return m


def small_2d(nx=40, ny=30, R=7.0, theta=60.0, tau=0.9, sigma=5e-3, xi=1.0, N=None, cx=None):
    N = N or int(round(2 * math.pi * R / 0.7))
    cx = nx / 2.0 + 0.37 if cx is None else cx
    nodes = W.circle(N, R, (cx, W.WALL_PLANE + R + 2 * xi))
    return W.Workload("small2d", 9, nx, ny, 1, tau, sigma, xi, theta, 9, 3, 100, nodes, None)


def small_3d(n=24, nz=20, R=6.0, level=2, theta=75.0, tau=0.8, sigma=5e-3, xi=1.0):
    nodes, faces = W.icosphere(level, R, (n / 2.0 + 0.31, n / 2.0 - 0.22, W.WALL_PLANE + R + 2 * xi))
    return W.Workload("small3d", 19, n, n, nz, tau, sigma, xi, theta, 9, 3, 100, nodes, faces)
