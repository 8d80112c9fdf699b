"""Pins of the oracle's viscosity-ratio step (Sec. 2): fluid nodes inside the
interface relax with tau (tau_in), those outside with tau_out, the two sets
found by ray tracing along the lattice columns.

The classification is checked against independent definitions: a winding
number (angle sum) for a non-convex 2D polygon, the box and the sphere
inequalities for 3D meshes.  The relaxation-time assignment is checked by the
decay rate of a shear wave, nu k^2 with nu = (tau - 1/2)/3, in a box that a
passive ring encloses completely (tau_in) or that holds no interface
(tau_out); tau_out = tau reproduces the single-tau run exactly.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import workloads as W
from helpers import box_mesh, star


def winding_inside(poly, x, y):
    """Independent point-in-polygon: total turning angle of the polygon seen
    from (x, y) is 2 pi inside and 0 outside."""
    d = poly - np.array([x, y])
    a = np.arctan2(d[:, 1], d[:, 0])
    da = np.diff(np.concatenate([a, a[:1]]))
    da = (da + np.pi) % (2 * np.pi) - np.pi
    return abs(da.sum()) > np.pi


def test_classification_star_polygon_2d():
    nx, ny = 48, 40
    poly = star(5, 6.3, 15.1, np.array([23.37, 19.61]))
    s = oracle.Sim(9, nx, ny, walls=False, wetting=False, tau=0.8, tau_out=1.1)
    s.set_interface(poly)
    m = s.inside_mask()[0]
    for y in range(ny):
        for x in range(nx):
            assert bool(m[y, x]) == winding_inside(poly, x, y), (x, y)
    assert 0 < m.sum() < nx * ny


def test_classification_box_3d():
    nx, ny, nz = 16, 14, 12
    v, tri = box_mesh((3.3, 2.6, 1.7), (11.2, 9.4, 8.8))
    s = oracle.Sim(19, nx, ny, nz, walls=False, wetting=False, tau=0.8, tau_out=1.1)
    s.set_interface(v, tri)
    m = s.inside_mask()
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    expect = (x > 3.3) & (x < 11.2) & (y > 2.6) & (y < 9.4) & (z > 1.7) & (z < 8.8)
    assert np.array_equal(m.astype(bool), expect)


def test_classification_sphere_3d():
    R, c = 7.3, np.array([12.21, 11.87, 10.63])
    q, tri = W.icosphere(4, R, tuple(c))
    s = oracle.Sim(19, 24, 24, 22, walls=False, wetting=False, tau=0.8, tau_out=1.1)
    s.set_interface(q, tri)
    m = s.inside_mask().astype(bool)
    z, y, x = np.mgrid[0:22, 0:24, 0:24]
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    sure = np.abs(r - R) > 0.3
    assert np.array_equal(m[sure], (r < R)[sure])


def shear_wave_rate(tau_in, tau_out, ring, nx=8, ny=32, steps=(300, 1500)):
    """Decay rate of u_x = U sin(2 pi y / ny) in a periodic box."""
    Q = 9
    U = 1e-4
    k = 2 * math.pi / ny
    s = oracle.Sim(Q, nx, ny, walls=False, wetting=False, sigma=0.0, tau=tau_in, tau_out=tau_out)
    f = np.zeros((Q, 1, ny, nx))
    for y in range(ny):
        f[:, 0, y, :] = oracle.equilibrium(Q, 1.0, [U * math.sin(k * y), 0.0, 0.0])[:, None]
    s.set_populations(f)
    if ring:
        # a passive rectangle (sigma = 0) enclosing every cell of the box; its
        # horizontal edges sit where the wave has no velocity
        xs = np.arange(-0.4, nx - 0.4, 0.5)
        ys = np.arange(-0.3, ny - 0.7, 0.5)
        bottom = np.stack([xs, np.full_like(xs, -0.3)], 1)
        right = np.stack([np.full_like(ys, nx - 0.4), ys], 1)
        top = np.stack([xs[::-1] + 0.5, np.full_like(xs, ny - 0.7)], 1)
        left = np.stack([np.full_like(ys, -0.4), ys[::-1] + 0.5], 1)
        s.set_interface(np.concatenate([bottom, right, top, left]))
        assert s.inside_mask().all()

    def amp():
        _, u, _ = s.fields()
        prof = u[0, 0, :, :].mean(axis=1)
        return 2.0 / ny * np.sum(prof * np.sin(k * np.arange(ny)))

    s.step(steps[0])
    a0 = amp()
    s.step(steps[1] - steps[0])
    a1 = amp()
    s.close()
    return -math.log(a1 / a0) / (steps[1] - steps[0]), k


@pytest.mark.parametrize("tau_in,tau_out", [(0.7, 1.2), (1.3, 0.6)])
def test_relaxation_times_by_region(tau_in, tau_out):
    rate_in, k = shear_wave_rate(tau_in, tau_out, ring=True)
    rate_out, _ = shear_wave_rate(tau_in, tau_out, ring=False)
    nu_in, nu_out = (tau_in - 0.5) / 3, (tau_out - 0.5) / 3
    assert abs(rate_in / (nu_in * k * k) - 1) < 0.01
    assert abs(rate_out / (nu_out * k * k) - 1) < 0.01


def test_equal_relaxation_times_reduce_to_single_tau():
    wl = W.drop_2d_128x64()
    a = oracle.Sim(9, wl.nx, wl.ny, tau=1.0, sigma=wl.sigma, xi=wl.xi, theta_eq_deg=60.0)
    b = oracle.Sim(9, wl.nx, wl.ny, tau=1.0, sigma=wl.sigma, xi=wl.xi, theta_eq_deg=60.0,
                   tau_out=1.0)
    for s in (a, b):
        s.set_interface(wl.nodes)
        s.step(50)
    assert np.array_equal(a.populations(), b.populations())
