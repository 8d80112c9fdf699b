"""Pins of the oracle's drop-in-shear pieces (Sec. 4): moving-wall bounce-back,
equilibrium initialisation from fields, and the deformation index D (Eq. 15).

- Plane Couette flow between walls moving at u_lo and u_hi is an exact
  steady solution of BGK with halfway bounce-back: u(a) = u_lo + (u_hi -
  u_lo) (a - 1/2) / (L - 2) on the fluid layers a = 1 .. L-2 (wall planes at
  1/2 and L - 3/2), for any tau.  A sign error or a missing factor in the
  wall term changes the slope or the offset.
- Walls moving together carry the fluid as a plug.
- f_eq(rho, u) has moments rho and rho u (Eq. 3), for the cells set.
- D, r1, r3 and the inclination of a linearly stretched and rotated sphere
  or circle are those of the ellipsoid / ellipse (a regular polygon and an
  icosphere have isotropic second moments, so the linear map carries them
  exactly); a star-shaped ring is checked against brute-force moments
  sampled on a fine grid.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import workloads as W


def couette_profile(u_lo, u_hi, L):
    a = np.arange(1, L - 1)
    return u_lo + (u_hi - u_lo) * (a - 0.5) / (L - 2)


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_couette_2d(tau):
    ny = 14
    s = oracle.Sim(9, 3, ny, tau=tau, wetting=False, sigma=0.0,
                   wall_u_lo=(-0.01, 0.0), wall_u_hi=(0.02, 0.0))
    n = int(40 * (ny - 2) ** 2 / ((tau - 0.5) / 3.0) / math.pi ** 2)
    s.step(n)
    rho, u, _ = s.fields()
    expect = couette_profile(-0.01, 0.02, ny)
    for x in range(3):
        assert np.max(np.abs(u[0, 0, 1:-1, x] - expect)) < 1e-13
        assert np.max(np.abs(u[1, 0, 1:-1, x])) < 1e-14
        # rho stays 1 up to the rounding of the raw populations, which drifts
        # by about 1e-16 per step once the fluid moves (linear in the step
        # count, independent of the wall speed)
        assert np.max(np.abs(rho[0, 1:-1, x] - 1.0)) < 1e-15 * n
    s.close()


def test_couette_3d_two_components():
    nz = 12
    s = oracle.Sim(19, 3, 4, nz, tau=0.9, wetting=False, sigma=0.0,
                   wall_u_lo=(0.01, -0.005, 0.0), wall_u_hi=(-0.02, 0.015, 0.0))
    s.step(int(40 * (nz - 2) ** 2 / (0.4 / 3.0) / math.pi ** 2))
    _, u, _ = s.fields()
    for k, (lo, hi) in enumerate([(0.01, -0.02), (-0.005, 0.015)]):
        prof = u[k, 1:-1, :, :]
        expect = couette_profile(lo, hi, nz)[:, None, None]
        assert np.max(np.abs(prof - expect)) < 1e-13
    assert np.max(np.abs(u[2, 1:-1])) < 1e-14
    s.close()


def test_walls_moving_together_give_plug_flow():
    s = oracle.Sim(9, 4, 10, tau=0.8, wetting=False, sigma=0.0,
                   wall_u_lo=(0.03, 0.0), wall_u_hi=(0.03, 0.0))
    s.step(3000)
    _, u, _ = s.fields()
    assert np.max(np.abs(u[0, 0, 1:-1, :] - 0.03)) < 1e-12
    s.close()


def test_moving_walls_conserve_mass_with_a_drop():
    wl = W.drop_2d_128x64()
    s = oracle.Sim(9, wl.nx, wl.ny, tau=1.0, sigma=wl.sigma, xi=wl.xi, wetting=False,
                   wall_u_lo=(-0.002, 0.0), wall_u_hi=(0.002, 0.0))
    s.set_interface(wl.nodes)
    f0 = s.populations()
    fluid = np.ones(f0.shape[1:], dtype=bool)
    fluid[:, 0, :] = fluid[:, -1, :] = False
    mass0 = f0[:, fluid].sum()
    s.step(200)
    f1 = s.populations()
    assert abs(f1[:, fluid].sum() - mass0) < 1e-10 * mass0
    s.close()


def test_set_equilibrium_moments():
    rng = np.random.default_rng(5)
    for Q, dims in ((9, (7, 5, 1)), (19, (5, 4, 3))):
        nx, ny, nz = dims
        s = oracle.Sim(Q, nx, ny, nz, walls=False, wetting=False, sigma=0.0)
        dim = 2 if Q == 9 else 3
        rho = 1.0 + 0.05 * rng.standard_normal((nz, ny, nx))
        u = 0.05 * rng.standard_normal((dim, nz, ny, nx))
        s.set_equilibrium(u, rho)
        f = s.populations()
        c, w, _ = oracle.lattice(Q)
        assert np.allclose(f.sum(axis=0), rho, rtol=0, atol=1e-14)
        for k in range(dim):
            mom = np.tensordot(c[:, k].astype(float), f, axes=(0, 0))
            assert np.allclose(mom, rho * u[k], rtol=0, atol=1e-14)
        # second moment of f_eq: rho (u u + c_s^2 I)
        pxx = np.tensordot((c[:, 0] * c[:, 0]).astype(float), f, axes=(0, 0))
        assert np.allclose(pxx, rho * (u[0] * u[0] + 1.0 / 3.0), rtol=0, atol=1e-14)
        s.close()


@pytest.mark.parametrize("axes,angle", [((12.0, 9.0, 7.0), 20.0), ((8.0, 8.0, 11.0), -35.0)])
def test_deformation_of_an_ellipsoid(axes, angle):
    q, tri = W.icosphere(4, 1.0, (0.0, 0.0, 0.0))
    q = q * np.array(axes)
    th = math.radians(angle)
    Rm = np.array([[math.cos(th), 0, -math.sin(th)], [0, 1, 0], [math.sin(th), 0, math.cos(th)]])
    q = q @ Rm.T + np.array([31.3, 17.2, 25.9])
    d = oracle.deformation(q, tri)
    a, c = axes[0], axes[2]
    r1, r3 = max(a, c), min(a, c)
    # the mesh is inscribed, so r's are slightly short; their ratio is exact
    assert abs(d["D"] - (r1 - r3) / (r1 + r3)) < 1e-12
    assert abs(d["r1"] / d["r3"] - r1 / r3) < 1e-12
    assert abs(d["r1"] - r1) < 0.01 * r1
    major = angle if a > c else angle + 90.0
    major = (major + 90.0) % 180.0 - 90.0
    assert abs(d["angle_deg"] - major) < 1e-9


def test_deformation_of_a_sphere_and_an_ellipse():
    q, tri = W.icosphere(3, 19.0, (40.0, 40.0, 40.0))
    assert abs(oracle.deformation(q, tri)["D"]) < 1e-13
    t = np.linspace(0, 2 * math.pi, 301, endpoint=False)
    th = math.radians(-28.0)
    e = np.stack([10.0 * np.cos(t), 6.0 * np.sin(t)], 1)
    e = e @ np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]]).T + 50.0
    d = oracle.deformation(e)
    assert abs(d["D"] - 4.0 / 16.0) < 1e-12
    assert abs(d["angle_deg"] - (-28.0)) < 1e-9


def test_deformation_brute_force_moments_irregular_ring():
    # a radial function with no rotational symmetry (non-convex in places)
    t = np.linspace(0, 2 * math.pi, 240, endpoint=False)
    r = 9.0 + 2.5 * np.sin(2 * t + 0.3) + 1.5 * np.cos(3 * t) + 0.8 * np.sin(5 * t + 1.1)
    poly = np.stack([r * np.cos(t) + 0.37, r * np.sin(t) - 0.21], 1)
    d = oracle.deformation(poly)
    h = 0.02
    xs = np.arange(-15.0, 15.0, h) + h / 2
    X, Y = np.meshgrid(xs, xs)
    # even-odd rule by crossings of horizontal rays (independent of the oracle)
    inside = np.zeros_like(X, dtype=bool)
    n = len(poly)
    for j in range(n):
        (x0, y0), (x1, y1) = poly[j], poly[(j + 1) % n]
        if y0 == y1:
            continue
        cond = (Y >= min(y0, y1)) & (Y < max(y0, y1))
        xc = x0 + (Y - y0) * (x1 - x0) / (y1 - y0)
        inside ^= cond & (X < xc)
    A = inside.sum() * h * h
    gx, gy = X[inside].mean(), Y[inside].mean()
    sxx = ((X[inside] - gx) ** 2).sum() * h * h
    syy = ((Y[inside] - gy) ** 2).sum() * h * h
    sxy = ((X[inside] - gx) * (Y[inside] - gy)).sum() * h * h
    mean, rad = 0.5 * (sxx + syy), math.hypot(0.5 * (sxx - syy), sxy)
    r1, r3 = math.sqrt(4 * (mean + rad) / A), math.sqrt(4 * (mean - rad) / A)
    assert abs(d["volume"] - A) < 2e-3 * A
    assert abs(d["r1"] - r1) < 2e-3 * r1 and abs(d["r3"] - r3) < 2e-3 * r3
    ang = 0.5 * math.degrees(math.atan2(2 * sxy, sxx - syy))
    assert abs(d["angle_deg"] - ang) < 0.5
