"""Pins of the oracle's interface mechanics (A1) and IB coupling (A2, A5).

Surface tension is checked against a finite-difference gradient of the
interface length / area (computed here from the definition of the measure,
not from the oracle), closed forms on regular polygons, and the invariances
that make the total force and torque vanish.  The wetting force is checked on
flat pieces of interface where n, chi and d are known by construction.  The
spread and interpolation operators (Eq. 7-8) are checked for adjointness,
the partition of unity and first-moment conditions, and exactness on linear
fields.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import workloads as W


def perimeter(q):
    return np.linalg.norm(np.roll(q, -1, axis=0) - q, axis=1).sum()


def surface_area(q, tri):
    a, b, c = q[tri[:, 0]], q[tri[:, 1]], q[tri[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum()


def fd_gradient(fun, q, h=1e-6):
    g = np.zeros_like(q)
    for idx in np.ndindex(*q.shape):
        qp = q.copy()
        qm = q.copy()
        qp[idx] += h
        qm[idx] -= h
        g[idx] = (fun(qp) - fun(qm)) / (2 * h)
    return g


def test_tension_2d_is_minus_sigma_grad_length():
    rng = np.random.default_rng(10)
    q = W.circle(24, 7.0, (20.0, 15.0)) + rng.uniform(-0.3, 0.3, (24, 2))
    sigma = 0.013
    out = oracle.nodal_forces(q, sigma=sigma)
    g = fd_gradient(perimeter, q)
    assert np.allclose(out["phi_sigma"], -sigma * g, atol=1e-9)
    assert np.allclose(out["phi"], out["phi_sigma"])  # no wetting requested


def test_tension_3d_is_minus_sigma_grad_area():
    rng = np.random.default_rng(11)
    q, tri = W.icosphere(1, 5.0, (10.0, 10.0, 10.0))
    q = q + rng.uniform(-0.2, 0.2, q.shape)
    sigma = 0.02
    out = oracle.nodal_forces(q, tri, sigma=sigma)
    g = fd_gradient(lambda x: surface_area(x, tri), q)
    assert np.allclose(out["phi_sigma"], -sigma * g, atol=1e-8)


@pytest.mark.parametrize("N", [3, 8, 50, 200])
def test_regular_polygon_closed_form(N):
    R, sigma = 20.0, 1e-3
    c = np.array([64.0, 22.5])
    q = W.circle(N, R, c)
    out = oracle.nodal_forces(q, sigma=sigma)
    radial = (q - c) / R
    mag = np.linalg.norm(out["phi"], axis=1)
    assert np.allclose(mag, 2 * sigma * math.sin(math.pi / N), rtol=1e-12)
    # directed radially inward
    assert np.allclose(out["phi"] / mag[:, None], -radial, atol=1e-12)
    # node normal is the outward radial direction, 1-ring length = 2 * side
    assert np.allclose(out["normal"], radial, atol=1e-12)
    assert np.allclose(out["chi"], 2 * 2 * R * math.sin(math.pi / N), rtol=1e-12)


def test_tension_free_of_net_force_and_torque():
    rng = np.random.default_rng(12)
    q2 = W.circle(40, 9.0, (30.0, 30.0)) + rng.uniform(-0.5, 0.5, (40, 2))
    f2 = oracle.nodal_forces(q2, sigma=0.1)["phi_sigma"]
    assert np.allclose(f2.sum(0), 0, atol=1e-15)
    assert abs(np.sum(q2[:, 0] * f2[:, 1] - q2[:, 1] * f2[:, 0])) < 1e-13
    q3, tri = W.icosphere(2, 6.0, (12.0, 12.0, 12.0))
    q3 = q3 + rng.uniform(-0.3, 0.3, q3.shape)
    f3 = oracle.nodal_forces(q3, tri, sigma=0.1)["phi_sigma"]
    assert np.allclose(f3.sum(0), 0, atol=1e-14)
    assert np.allclose(np.cross(q3, f3).sum(0), 0, atol=1e-12)


def test_icosphere_laplace_force_and_measures():
    R, sigma = 40.0, 1e-3
    q, tri = W.icosphere(5, R, (128.0, 128.0, 42.5))
    out = oracle.nodal_forces(q, tri, sigma=sigma)
    # sum of 1-ring areas = 3 x total area; area close to 4 pi R^2
    A = surface_area(q, tri)
    assert math.isclose(out["chi"].sum(), 3 * A, rel_tol=1e-12)
    assert abs(A / (4 * math.pi * R * R) - 1) < 5e-3
    radial = (q - np.array([128.0, 128.0, 42.5])) / R
    assert np.max(np.linalg.norm(out["normal"] - radial, axis=1)) < 5e-3
    # normal force density ~ Laplace: phi . n ~ -sigma (2 / R) chi / 3
    fn = np.einsum("ij,ij->i", out["phi"], out["normal"])
    expect = -sigma * (2.0 / R) * out["chi"] / 3.0
    assert abs(fn.sum() / expect.sum() - 1) < 1e-2


def test_wetting_force_flat_bottom_2d():
    # rectangle ring, CCW, bottom edge at height y0 with spacing h
    h, y0, sigma, xi, A = 0.5, 2.0, 1e-3, 1.0, 4e-3
    xs = np.arange(0, 10.0 + 1e-9, h)
    bottom = np.stack([xs, np.full_like(xs, y0)], 1)
    ys = np.arange(y0 + h, y0 + 6.0 + 1e-9, h)
    right = np.stack([np.full_like(ys, 10.0), ys], 1)
    top = np.stack([xs[::-1][1:], np.full(len(xs) - 1, ys[-1])], 1)
    left = np.stack([np.zeros(len(ys) - 2), ys[::-1][1:-1]], 1)
    q = np.concatenate([bottom, right, top, left])
    out = oracle.nodal_forces(q, sigma=sigma, wetting=True, A=A, xi=xi, n=9, m=3, wall_plane=0.5)
    d = y0 - 0.5
    pi = A * ((xi / d) ** 9 - (xi / d) ** 3)
    for j in range(2, len(xs) - 2):   # interior bottom nodes
        assert np.allclose(out["normal"][j], [0.0, -1.0], atol=1e-15)
        assert math.isclose(out["chi"][j], 2 * h, rel_tol=1e-14)
        # -chi Pi n / 2 = (0, h Pi)
        assert np.allclose(out["phi_pi"][j], [0.0, h * pi], atol=1e-18)
        assert np.allclose(out["phi_sigma"][j], 0.0, atol=1e-18)
    assert not out["bad"]
    q_in = q.copy()
    q_in[0, 1] = 0.4
    assert oracle.nodal_forces(q_in, sigma=sigma, wetting=True, A=A, xi=xi)["bad"]


def test_wetting_force_flat_bottom_3d():
    # a flat triangulated square patch at height z0 (faces oriented downward,
    # as the bottom of a drop): interior nodes have n = -z, chi = 6 tri areas
    h, z0, xi, A = 1.0, 1.7, 1.0, 2e-3
    n = 6
    P = np.array([[i * h, j * h, z0] for j in range(n) for i in range(n)])
    tri = []
    for j in range(n - 1):
        for i in range(n - 1):
            a, b, c, d = j * n + i, j * n + i + 1, (j + 1) * n + i, (j + 1) * n + i + 1
            tri += [(a, c, b), (b, c, d)]   # normal -z
    tri = np.array(tri, dtype=np.int32)
    out = oracle.nodal_forces(P, tri, sigma=0.0, wetting=True, A=A, xi=xi, wall_plane=0.5)
    pi = A * ((xi / (z0 - 0.5)) ** 9 - (xi / (z0 - 0.5)) ** 3)
    j = 2 * n + 2
    assert np.allclose(out["normal"][j], [0, 0, -1], atol=1e-15)
    assert math.isclose(out["chi"][j], 6 * 0.5 * h * h, rel_tol=1e-14)
    assert np.allclose(out["phi_pi"][j], [0, 0, 6 * 0.5 * h * h * pi / 3], atol=1e-18)


def _sim(Q, nx, ny, nz=1, walls=False, **kw):
    return oracle.Sim(Q, nx, ny, nz, walls=walls, wetting=False, **kw)


@pytest.mark.parametrize("Q,shape", [(9, (20, 16, 1)), (19, (12, 10, 9))])
def test_spread_interp_adjoint_and_moments(Q, shape):
    nx, ny, nz = shape
    dim = 2 if Q == 9 else 3
    s = _sim(Q, nx, ny, nz)
    rng = np.random.default_rng(13)
    N = 17
    # nodes away from the periodic seam so that first moments need no unwrapping
    lo, hi = 3.0, np.array([nx, ny, nz][:dim]) - 4.0
    q = rng.uniform(lo, hi, (N, dim))
    s.set_interface(q, None if dim == 2 else np.zeros((0, 3), np.int32))
    phi = rng.normal(size=(N, dim))
    F = s.spread(phi)
    Fk = F[:dim].reshape(dim, -1)
    # partition of unity: total spread force = total nodal force
    assert np.allclose(Fk.sum(1), phi.sum(0), atol=1e-12)
    # first moment: sum_x x F(x) = sum_j q_j phi_j (tensor form)
    grids = np.meshgrid(*[np.arange(n) for n in (nz, ny, nx)], indexing="ij")
    coords = [grids[2].ravel(), grids[1].ravel(), grids[0].ravel()][:dim]
    mom = np.array([[np.sum(coords[a] * Fk[b]) for b in range(dim)] for a in range(dim)])
    assert np.allclose(mom, q.T @ phi, atol=1e-10)
    # adjointness with interpolation: <F, u> = <phi, qdot>
    u = rng.normal(size=(3,) + s.shape)
    if dim == 2:
        u[2] = 0.0
    qd = s.interpolate(u)
    lhs = np.sum(F[:dim] * u[:dim])
    rhs = np.sum(phi * qd)
    assert math.isclose(lhs, rhs, rel_tol=1e-12, abs_tol=1e-12)
    # linear velocity fields are interpolated exactly
    a = rng.normal(size=dim)
    B = rng.normal(size=(dim, dim))
    ulin = np.zeros((3,) + s.shape)
    for k in range(dim):
        ulin[k] = a[k] + sum(B[k, m] * coords[m].reshape(s.shape) for m in range(dim))
    qd = s.interpolate(ulin)
    assert np.allclose(qd, a[None, :] + q @ B.T, atol=1e-12)
    s.close()


def test_spread_discards_solid_layers():
    s = oracle.Sim(9, 16, 12, walls=True, wetting=False)
    q = np.array([[7.3, 1.2]])   # stencil rows 0..3: row 0 is solid
    s.set_interface(q)
    F = s.spread(np.array([[0.0, 1.0]]))
    assert np.all(F[:, :, 0, :] == 0.0)
    wy = sum(oracle.delta4(1.2 - j) for j in (1, 2, 3))
    assert wy < 1.0
    assert math.isclose(F[1].sum(), wy, rel_tol=1e-14)
    # interpolation sees zero velocity on solid layers
    u = np.ones((3,) + s.shape)
    qd = s.interpolate(u)
    assert math.isclose(qd[0, 0], wy, rel_tol=1e-14)
    s.close()


def test_spread_discards_layers_outside_lattice():
    s = oracle.Sim(9, 16, 12, walls=True, wetting=False)
    s.set_interface(np.array([[7.3, 0.7]]))   # stencil rows -1..2: rows -1 and 0 dropped
    F = s.spread(np.array([[0.0, 1.0]]))
    wy = sum(oracle.delta4(0.7 - j) for j in (1, 2))
    assert math.isclose(F[1].sum(), wy, rel_tol=1e-14)
    s.close()
