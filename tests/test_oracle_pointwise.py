"""Pins of the oracle's pointwise pieces against what the mathematics fixes.

Lattice isotropy, the moments of the equilibrium (Eq. 3) and of the Guo source
(Eq. 4), the Peskin 4-point delta conditions, and the wetting potential
(Eq. 10) with its amplitude (Eq. 11).  None of these retype the oracle's
formulas: they check the moment identities those formulas must satisfy.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

CS2 = 1.0 / 3.0


@pytest.mark.parametrize("Q", [9, 19])
def test_lattice_isotropy(Q):
    c, w, opp = oracle.lattice(Q)
    dim = 2 if Q == 9 else 3
    assert len(set(map(tuple, c))) == Q
    assert np.all(c[opp] == -c)
    assert abs(w.sum() - 1.0) < 1e-15
    d = np.eye(3)[:dim, :dim]
    cc = c[:, :dim].astype(float)
    # odd moments vanish, even moments are isotropic with cs^2 = 1/3
    assert np.allclose(np.einsum("i,ia->a", w, cc), 0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, cc, cc), CS2 * d, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, cc, cc, cc), 0, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, cc, cc, cc, cc)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, iso, atol=1e-15)
    if dim == 2:
        assert np.all(c[:, 2] == 0)


@pytest.mark.parametrize("Q", [9, 19])
def test_equilibrium_moments(Q):
    c, w, _ = oracle.lattice(Q)
    dim = 2 if Q == 9 else 3
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(0.8, 1.2)
        u = np.zeros(3)
        u[:dim] = rng.uniform(-0.1, 0.1, dim)
        feq = oracle.equilibrium(Q, rho, u)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.allclose(c.T @ feq, rho * u, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", feq, c, c)
        expect = rho * CS2 * np.diag([1.0] * dim + [0.0] * (3 - dim)) + rho * np.outer(u, u)
        assert np.allclose(P, expect, atol=1e-14)
    # rest state: feq(1, 0) = w
    assert np.allclose(oracle.equilibrium(Q, 1.0, [0, 0, 0]), w, atol=0)


@pytest.mark.parametrize("Q", [9, 19])
def test_guo_source_moments(Q):
    c, w, _ = oracle.lattice(Q)
    dim = 2 if Q == 9 else 3
    rng = np.random.default_rng(2)
    for tau in (0.55, 0.8, 1.0, 1.7):
        for _ in range(10):
            u = np.zeros(3)
            F = np.zeros(3)
            u[:dim] = rng.uniform(-0.1, 0.1, dim)
            F[:dim] = rng.uniform(-1e-3, 1e-3, dim)
            S = oracle.guo_source(Q, tau, u, F)
            pref = 1.0 - 1.0 / (2.0 * tau)
            assert abs(S.sum()) < 1e-17
            assert np.allclose(c.T @ S, pref * F, atol=1e-18)
            P = np.einsum("i,ia,ib->ab", S, c, c)
            assert np.allclose(P, pref * (np.outer(u, F) + np.outer(F, u)), atol=1e-18)


def test_delta4_conditions():
    # discrete partition of unity, zero first moment, sum of squares 3/8
    rng = np.random.default_rng(3)
    for r in np.concatenate([rng.uniform(-3, 3, 200), [0.0, 0.5, 1.0, 1.5, 2.0, -1.0]]):
        base = math.floor(r) - 3
        pts = np.arange(base, base + 8)
        phi = np.array([oracle.delta4(r - i) for i in pts])
        assert abs(phi.sum() - 1.0) < 1e-14
        assert abs(((r - pts) * phi).sum()) < 1e-14
        assert abs((phi ** 2).sum() - 3.0 / 8.0) < 1e-14
        assert np.all(phi >= 0)
        # even/odd split: sum over even points = sum over odd points = 1/2
        even = phi[(pts % 2) == 0].sum()
        assert abs(even - 0.5) < 1e-14
    assert oracle.delta4(0.0) == 0.5
    assert abs(oracle.delta4(1.0) - 0.25) < 1e-16
    assert oracle.delta4(2.0) == 0.0
    assert oracle.delta4(2.5) == 0.0
    assert oracle.delta4(-0.3) == oracle.delta4(0.3)


def test_wetting_amplitude_closed_forms():
    # Eq. 11 with (n, m) = (9, 3): (m-1)(n-1)/(n-m) = 16/6
    s, xi = 1e-3, 2.0
    assert math.isclose(oracle.wetting_A(s, xi, 60.0, 9, 3), s * 16 / 6 / xi * 1.5, rel_tol=1e-15)
    assert math.isclose(oracle.wetting_A(s, xi, 90.0, 9, 3), s * 16 / 6 / xi, rel_tol=1e-15)
    assert abs(oracle.wetting_A(s, xi, 180.0, 9, 3)) < 1e-19
    # (n, m) = (4, 2): (1)(3)/(2) = 1.5
    assert math.isclose(oracle.wetting_A(1.0, 1.0, 0.0, 4, 2), 3.0, rel_tol=1e-15)
    # more wetting (smaller angle) -> larger amplitude
    a = [oracle.wetting_A(s, xi, t, 9, 3) for t in (30, 60, 90, 120, 150)]
    assert all(x > y for x, y in zip(a, a[1:]))


def test_wetting_potential():
    A, xi = 0.7, 1.5
    assert oracle.wetting_Pi(A, xi, 9, 3, xi) == 0.0
    # d = xi / 2: A (2^9 - 2^3)
    assert math.isclose(oracle.wetting_Pi(A, xi, 9, 3, xi / 2), A * (512 - 8), rel_tol=1e-15)
    # d = 2 xi: A (2^-9 - 2^-3)
    assert math.isclose(oracle.wetting_Pi(A, xi, 9, 3, 2 * xi), A * (2 ** -9 - 2 ** -3),
                        rel_tol=1e-15)
    # repulsive below xi, attractive above, decaying as d^-m
    assert oracle.wetting_Pi(A, xi, 9, 3, 0.9 * xi) > 0
    assert oracle.wetting_Pi(A, xi, 9, 3, 1.1 * xi) < 0
    far = [oracle.wetting_Pi(A, xi, 9, 3, d) * d ** 3 for d in (50.0, 100.0)]
    assert math.isclose(far[0], far[1], rel_tol=1e-9)
