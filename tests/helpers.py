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


def star(n_arms, r_in, r_out, centre, per_arm=24, phase=0.17):
    pts = []
    for k in range(n_arms * 2):
        r0 = r_out if k % 2 == 0 else r_in
        r1 = r_in if k % 2 == 0 else r_out
        a0 = phase + math.pi * k / n_arms
        a1 = phase + math.pi * (k + 1) / n_arms
        for t in np.linspace(0, 1, per_arm, endpoint=False):
            p0 = np.array([r0 * math.cos(a0), r0 * math.sin(a0)])
            p1 = np.array([r1 * math.cos(a1), r1 * math.sin(a1)])
            pts.append(centre + (1 - t) * p0 + t * p1)
    return np.array(pts)


def box_mesh(lo, hi):
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]])
    quads = [(0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)]
    tri = []
    for a, b, c, d in quads:   # outward orientation
        tri += [(a, b, c), (a, c, d)]
    return v, np.array(tri, dtype=np.int32)
