"""The seeded input generators: closed, outward-oriented meshes of the sizes
the workloads name, and shapes with the stated geometry (CPU only)."""
import math
from collections import Counter

import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import workloads as W


def mesh_checks(q, tri):
    """Closed 2-manifold, consistently oriented, outward (positive volume)."""
    E = Counter()
    for a, b, c in tri:
        for u, v in ((a, b), (b, c), (c, a)):
            E[(int(u), int(v))] += 1
    assert max(E.values()) == 1
    assert all((v, u) in E for (u, v) in E)
    V, F = len(q), len(tri)
    assert V - len(E) // 2 + F == 2          # Euler characteristic of a sphere
    a, b, c = q[tri[:, 0]], q[tri[:, 1]], q[tri[:, 2]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0


@pytest.mark.parametrize("freq", [1, 2, 5, 12])
def test_geodesic_sphere_counts_and_closure(freq):
    q, tri = W.geodesic_sphere(freq, 3.0, (1.0, 2.0, 3.0))
    assert q.shape == (10 * freq * freq + 2, 3) and tri.shape == (20 * freq * freq, 3)
    vol = mesh_checks(q - np.array([1.0, 2.0, 3.0]), tri)
    assert 0 < vol < 4.0 / 3.0 * math.pi * 27.0
    assert np.allclose(np.linalg.norm(q - np.array([1.0, 2.0, 3.0]), axis=1), 3.0)


def test_geodesic_sphere_matches_one_midpoint_refinement():
    # frequency 2 cuts every face at its edge midpoints, as one level of the
    # icosphere does (deeper levels differ: the icosphere projects after each)
    q1, t1 = W.geodesic_sphere(2, 1.0, (0.0, 0.0, 0.0))
    q2, t2 = W.icosphere(1, 1.0, (0.0, 0.0, 0.0))
    a = np.sort(np.round(q1, 12).view("f8,f8,f8").ravel())
    b = np.sort(np.round(q2, 12).view("f8,f8,f8").ravel())
    assert np.array_equal(a, b)


def test_paper_scale_mesh_size():
    s = W.spread3d_cap(1.1, t_mu_count=1.0)
    assert len(s.work.faces) == 118580          # about the paper's 120 000 triangles
    vol = mesh_checks(s.work.nodes, s.work.faces)
    R0 = s.R0
    # R0 is the radius of the sphere of the same volume as the hemisphere
    assert abs(vol / (4.0 / 3.0 * math.pi * R0 ** 3) - 1.0) < 1e-3
    assert s.work.xi == pytest.approx(0.05 * R0)
    z = s.work.nodes[:, 2]
    Rh = 2.0 ** (1.0 / 3.0) * R0
    assert abs(z.min() - (W.WALL_PLANE + s.work.xi)) < 1e-12
    assert abs(z.max() - z.min() - Rh) < 1e-3 * Rh   # no mesh vertex sits exactly on the pole
    assert s.t_mu == pytest.approx((1.1 - 0.5) / 3.0 * R0 / s.work.sigma)


@pytest.mark.parametrize("theta0", [60.0, 90.0, 150.0])
def test_truncated_sphere_geometry(theta0):
    R = 10.0
    q, tri = W.truncated_sphere(12, R, theta0, 2.0, (20.0, 21.0))
    vol = mesh_checks(q, tri)
    th = math.radians(theta0)
    cap = math.pi * R ** 3 * (2.0 - 3.0 * math.cos(th) + math.cos(th) ** 3) / 3.0
    assert abs(vol / cap - 1.0) < 0.02
    # the oracle's estimator reads the construction angle back
    s = oracle.Sim(19, 40, 42, 30, xi=0.5, theta_eq_deg=theta0)
    s.set_interface(q, tri)
    assert abs(s.observables()["theta_deg"] - theta0) < 1.0
    s.close()


def test_shear_drop_parameters():
    c = W.shear_drop()
    nu = (c.tau_out - 0.5) / 3.0
    assert c.gamma_dot * c.R0 ** 2 / nu == pytest.approx(0.01)
    assert nu * c.gamma_dot * c.R0 / c.work.sigma == pytest.approx(0.05)
    assert c.d_inf() == pytest.approx(35.0 / 32.0 * 0.05)
    u = c.initial_velocity()
    H = c.height
    top, bottom = u[0, -2, 0, 0], u[0, 1, 0, 0]
    # the fluid layers next to the walls lie half a spacing inside the planes
    assert top - bottom == pytest.approx(c.gamma_dot * (H - 1.0))
    assert c.wall_u_hi[0] - c.wall_u_lo[0] == pytest.approx(c.gamma_dot * H)
