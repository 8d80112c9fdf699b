"""Pins of the oracle's observables (A7) on shapes known by construction.

The paper measures the drop height as the distance between the highest and
lowest interface nodes (Sec. 3); the contact-angle estimator (algebraic
circle / sphere fit through the nodes above 3 xi, cut with the plane at the
lowest node) is a reading.  On an exact circular cap (2D) and spherical cap
(3D) closed by a flat base at height eps above the wall plane, the fitted
angle, contact-line radius, film thickness, height, enclosed area / volume
must be the construction's, and the mass of the rest state is the fluid
cell count.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import workloads as W


def cap_2d(R, theta_deg, eps, xc, n=4000):
    return W.truncated_circle(n, R, theta_deg, W.WALL_PLANE + eps, xc)


@pytest.mark.parametrize("theta", [40.0, 75.0, 90.0, 120.0, 150.0])
def test_circle_cap_angle_2d(theta):
    R, eps, xi = 30.0, 0.9, 1.0
    s = oracle.Sim(9, 160, 80, tau=1.0, walls=True, wetting=True, xi=xi, theta_eq_deg=theta)
    q = cap_2d(R, theta, eps, 80.0)
    s.set_interface(q)
    o = s.observables()
    th = math.radians(theta)
    assert abs(o["theta_deg"] - theta) < 1e-6
    assert abs(o["r_cl"] - R * math.sin(th)) < 1e-6
    assert abs(o["radius"] - R) < 1e-9
    assert abs(o["d_min"] - eps) < 1e-12
    assert abs(o["film"] - eps) < 1e-12
    assert abs(o["height"] - R * (1 - math.cos(th))) < 1e-3
    # enclosed area of the polygon ~ circular segment area
    seg = R * R * (th - math.sin(th) * math.cos(th))
    assert abs(o["volume"] / seg - 1) < 1e-5
    # rest state: mass = number of fluid cells
    assert o["mass"] == pytest.approx(160 * 78, rel=1e-12)
    s.close()


def spherical_cap(R, theta_deg, eps, centre_xy, level=6):
    """Icosphere nodes cut to a cap: nodes below the base plane are projected
    onto it (a flat base); faces keep the sphere's connectivity."""
    th = math.radians(theta_deg)
    zc = W.WALL_PLANE + eps - R * math.cos(th)
    q, tri = W.icosphere(level, R, (centre_xy[0], centre_xy[1], zc))
    base = W.WALL_PLANE + eps
    q[:, 2] = np.maximum(q[:, 2], base)
    return q, tri


@pytest.mark.parametrize("theta", [60.0, 90.0, 130.0])
def test_sphere_cap_angle_3d(theta):
    R, eps, xi = 20.0, 0.8, 1.0
    s = oracle.Sim(19, 64, 64, 48, tau=1.0, walls=True, wetting=True, xi=xi, theta_eq_deg=theta)
    q, tri = spherical_cap(R, theta, eps, (32.0, 32.0), level=5)
    s.set_interface(q, tri)
    o = s.observables()
    th = math.radians(theta)
    # nodes above 3 xi lie exactly on the sphere: the fit recovers it
    assert abs(o["radius"] - R) < 1e-8
    assert abs(o["theta_deg"] - theta) < 1e-6
    assert abs(o["r_cl"] - R * math.sin(th)) < 1e-6
    assert abs(o["d_min"] - eps) < 1e-12
    assert abs(o["film"] - eps) < 1e-12
    # volume of the cap (divergence theorem on the mesh) ~ analytic cap volume
    h = R * (1 - math.cos(th))
    vcap = math.pi * h * h * (3 * R - h) / 3.0
    assert abs(o["volume"] / vcap - 1) < 5e-3
    s.close()
