"""Pins of the oracle's elastic interface (Skalak strain energy on linear
triangles; 2D rings in plane strain), against what the law and the mechanics
fix, not against a retyped formula:

- homogeneous deformations of a flat, irregularly triangulated patch give the
  closed-form energy per reference area for uniaxial plane strain,
  equibiaxial stretch, pure shear and simple shear, whatever rigid motion is
  applied to the reference or the deformed patch;
- the small-strain moduli are the published ones: area dilation modulus
  K = G_s (1 + 2C) and shear modulus G_s;
- the nodal force is minus the finite-difference gradient of the energy on
  irregular deformed meshes and rings;
- zero force on the reference shape, zero net force and torque;
- a uniformly stretched regular N-gon: every node pulled radially inward by
  2 T sin(pi/N), T = G_s (1 + C) lambda (lambda^2 - 1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import workloads as W


def rotation(seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3))
    Qm, R = np.linalg.qr(A)
    Qm = Qm * np.sign(np.diag(R))
    if np.linalg.det(Qm) < 0:
        Qm[:, 0] = -Qm[:, 0]
    return Qm


def flat_patch(n=7, seed=1):
    """Irregular triangulation of the unit square in the xy plane: a jittered
    grid, every cell split along a random diagonal, counter-clockwise seen
    from +z."""
    rng = np.random.default_rng(seed)
    xs = np.linspace(0.0, 1.0, n)
    pts = []
    for j in range(n):
        for i in range(n):
            p = np.array([xs[i], xs[j], 0.0])
            if 0 < i < n - 1 and 0 < j < n - 1:
                p[:2] += rng.uniform(-0.25, 0.25, 2) / (n - 1)
            pts.append(p)
    tri = []
    for j in range(n - 1):
        for i in range(n - 1):
            a, b, c, d = j * n + i, j * n + i + 1, (j + 1) * n + i + 1, (j + 1) * n + i
            if rng.uniform() < 0.5:
                tri += [(a, b, c), (a, c, d)]
            else:
                tri += [(a, b, d), (b, c, d)]
    return np.array(pts), np.array(tri, dtype=np.int32)


def deform(p, F2):
    """Apply the in-plane linear map F2 (2x2) to the xy coordinates."""
    out = p.copy()
    out[:, :2] = p[:, :2] @ np.asarray(F2).T
    return out


def patch_energy(F2, Gs, C, ref_motion=0, cur_motion=0):
    q0, tri = flat_patch()
    q = deform(q0, F2)
    if ref_motion:
        R = rotation(ref_motion)
        q0 = q0 @ R.T + np.array([0.3, -1.2, 2.5])
    if cur_motion:
        R = rotation(cur_motion + 100)
        q = q @ R.T + np.array([-4.0, 0.7, 1.1])
    ref = oracle.elastic_reference(q0, tri)
    E, f = oracle.elastic_forces(q, ref, tri, Gs=Gs, C=C)
    return E, f, ref


def test_reference_area_is_the_patch_area():
    _, _, ref = patch_energy(np.eye(2), 1.0, 0.0)
    assert abs(ref[:, 4].sum() - 1.0) < 1e-13


@pytest.mark.parametrize("Gs,C", [(1.0, 0.0), (0.37, 1.0), (2.5, 10.0)])
@pytest.mark.parametrize("motion", [(0, 0), (3, 0), (0, 5), (7, 11)])
def test_homogeneous_deformations_closed_forms(Gs, C, motion):
    lam = 1.23
    # uniaxial plane strain: lambda1 = lam, lambda2 = 1
    E, _, _ = patch_energy([[lam, 0], [0, 1]], Gs, C, *motion)
    assert abs(E - Gs / 4 * (1 + C) * (lam ** 2 - 1) ** 2) < 1e-12 * max(1.0, E)
    # equibiaxial: lambda1 = lambda2 = lam
    E, _, _ = patch_energy([[lam, 0], [0, lam]], Gs, C, *motion)
    want = Gs / 4 * (2 * (lam ** 2 - 1) ** 2 + C * (lam ** 4 - 1) ** 2)
    assert abs(E - want) < 1e-12 * max(1.0, want)
    # pure shear: lambda1 = lam, lambda2 = 1/lam (area kept, I2 = 0)
    E, _, _ = patch_energy([[lam, 0], [0, 1 / lam]], Gs, C, *motion)
    I1 = lam ** 2 + lam ** -2 - 2
    assert abs(E - Gs / 4 * (I1 ** 2 + 2 * I1)) < 1e-12
    # simple shear x -> x + g y: I1 = g^2, I2 = 0
    g = 0.31
    E, _, _ = patch_energy([[1, g], [0, 1]], Gs, C, *motion)
    assert abs(E - Gs / 4 * (g ** 4 + 2 * g ** 2)) < 1e-12


@pytest.mark.parametrize("C", [0.0, 0.5, 3.0])
def test_small_strain_moduli(C):
    Gs, eps = 0.8, 1e-4
    # equibiaxial: W -> K/2 alpha^2 with areal strain alpha ~ 2 eps
    E, _, _ = patch_energy([[1 + eps, 0], [0, 1 + eps]], Gs, C)
    alpha = (1 + eps) ** 2 - 1
    K = 2 * E / alpha ** 2
    assert abs(K / (Gs * (1 + 2 * C)) - 1) < 1e-3
    # pure shear with principal strains +-eps: W -> 2 G_s eps^2
    E, _, _ = patch_energy([[1 + eps, 0], [0, 1 / (1 + eps)]], Gs, C)
    assert abs(E / (2 * Gs * eps ** 2) - 1) < 1e-3


def fd_gradient(q, ref, tri, Gs, C, h=1e-6):
    g = np.zeros_like(q)
    for j in range(q.shape[0]):
        for k in range(q.shape[1]):
            qp, qm = q.copy(), q.copy()
            qp[j, k] += h
            qm[j, k] -= h
            g[j, k] = (oracle.elastic_forces(qp, ref, tri, Gs=Gs, C=C)[0] -
                       oracle.elastic_forces(qm, ref, tri, Gs=Gs, C=C)[0]) / (2 * h)
    return g


def test_mesh_force_is_minus_energy_gradient():
    rng = np.random.default_rng(4)
    q0, tri = W.icosphere(1, 3.0, (0.0, 0.0, 0.0))
    q0 = q0 + rng.uniform(-0.2, 0.2, q0.shape)       # irregular reference
    ref = oracle.elastic_reference(q0, tri)
    A = np.eye(3) + rng.uniform(-0.15, 0.15, (3, 3))  # general deformation
    q = q0 @ A.T + rng.uniform(-0.1, 0.1, q0.shape)
    for Gs, C in ((1.0, 0.0), (0.3, 2.0)):
        E, f = oracle.elastic_forces(q, ref, tri, Gs=Gs, C=C)
        g = fd_gradient(q, ref, tri, Gs, C)
        assert np.max(np.abs(f + g)) < 1e-7 * np.max(np.abs(f))
        assert np.max(np.abs(f.sum(axis=0))) < 1e-12 * np.max(np.abs(f))
        torque = np.cross(q, f).sum(axis=0)
        assert np.max(np.abs(torque)) < 1e-11 * np.max(np.abs(f)) * np.max(np.abs(q))


def test_ring_force_is_minus_energy_gradient():
    rng = np.random.default_rng(8)
    q0 = W.circle(23, 5.0, (10.0, 7.0)) + rng.uniform(-0.3, 0.3, (23, 2))
    ref = oracle.elastic_reference(q0)
    q = q0 @ np.array([[1.2, 0.1], [-0.05, 0.9]]).T + rng.uniform(-0.1, 0.1, q0.shape)
    E, f = oracle.elastic_forces(q, ref, Gs=0.7, C=1.5)
    g = fd_gradient(q, ref, None, 0.7, 1.5)
    assert np.max(np.abs(f + g)) < 1e-7 * np.max(np.abs(f))
    assert np.max(np.abs(f.sum(axis=0))) < 1e-13 * np.max(np.abs(f))


@pytest.mark.parametrize("dim", [2, 3])
def test_zero_force_on_the_reference(dim):
    if dim == 3:
        q0, tri = W.icosphere(2, 4.0, (1.0, 2.0, 3.0))
    else:
        q0, tri = W.circle(40, 6.0, (3.0, 4.0)), None
    ref = oracle.elastic_reference(q0, tri)
    E, f = oracle.elastic_forces(q0, ref, tri, Gs=1.0, C=2.0)
    assert abs(E) < 1e-13 and np.max(np.abs(f)) < 1e-13


@pytest.mark.parametrize("N", [12, 50])
def test_stretched_polygon_closed_form(N):
    r0, lam, Gs, C = 4.0, 1.1, 0.6, 0.8
    q0 = W.circle(N, r0, (0.0, 0.0))
    ref = oracle.elastic_reference(q0)
    q = lam * q0
    E, f = oracle.elastic_forces(q, ref, Gs=Gs, C=C)
    T = Gs * (1 + C) * lam * (lam ** 2 - 1)
    radial = (f * q).sum(axis=1) / np.linalg.norm(q, axis=1)
    assert np.allclose(radial, -2 * T * math.sin(math.pi / N), rtol=1e-12)
    tangential = f[:, 0] * (-q[:, 1]) + f[:, 1] * q[:, 0]
    assert np.max(np.abs(tangential)) < 1e-13
    seg0 = 2 * r0 * math.sin(math.pi / N)
    assert abs(E - N * seg0 * Gs / 4 * (1 + C) * (lam ** 2 - 1) ** 2) < 1e-12


def test_sim_adds_elastic_force_relative_to_the_interface_as_set():
    # at the interface as set, the elastic force vanishes: the nodal forces
    # equal those without elasticity; after a stretch they differ by exactly
    # the elastic force of the stretched shape
    q0, tri = W.icosphere(2, 4.0, (12.0, 12.0, 9.0))
    kw = dict(tau=0.9, walls=True, wetting=True, sigma=2e-3, xi=1.0, theta_eq_deg=70.0)
    a = oracle.Sim(19, 24, 24, 20, **kw)
    b = oracle.Sim(19, 24, 24, 20, shear_modulus=5e-3, skalak_c=1.0, **kw)
    for s in (a, b):
        s.set_interface(q0, tri)
    pa, pb = a.nodal_forces()[0], b.nodal_forces()[0]
    assert np.max(np.abs(pb - pa)) < 1e-16
    for s in (a, b):
        s.step(20)
    qb = b.fields()[2]
    ref = oracle.elastic_reference(q0, tri)
    _, fe = oracle.elastic_forces(qb, ref, tri, Gs=5e-3, C=1.0)
    a2 = oracle.Sim(19, 24, 24, 20, **kw)
    a2.set_interface(qb, tri)
    assert np.max(np.abs(b.nodal_forces()[0] - (a2.nodal_forces()[0] + fe))) < 1e-15
    assert np.max(np.abs(fe)) > 0
