"""Pins of the oracle's time stepping against what the method fixes.

Streaming is checked by propagating single populations (Eq. 1 with the
collision switched off by a huge tau), bounce-back by their return at the
wall; conservation of mass and momentum on a periodic box; the rest state as
a fixed point; the body-force Poiseuille profile, which BGK with halfway
bounce-back and Guo forcing reproduces to round-off at tau = 1/2 + sqrt(3/16);
the viscosity of that flow against the tau / mu pairs printed in the paper;
the Laplace pressure of a free droplet; and the wetting physics the paper
states (Sec. 2): a film of thickness ~ xi that vanishes linearly with xi, and
an apparent contact angle that follows theta_eq.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2604_17463_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def momentum(c, f):
    return c.T.astype(float) @ f.reshape(f.shape[0], -1).sum(axis=1)


def near_eq_populations(Q, shape, seed, amp=0.05):
    _, w, _ = oracle.lattice(Q)
    noise = W.random_perturbation((Q,) + shape, seed, amp)
    return w.reshape((Q,) + (1,) * len(shape)) * (1.0 + noise)


@pytest.mark.parametrize("Q,dims", [(9, (7, 6, 1)), (19, (5, 4, 6))])
@pytest.mark.parametrize("walls", [False, True])
def test_streaming_moves_single_populations(Q, dims, walls):
    c, w, opp = oracle.lattice(Q)
    nx, ny, nz = dims
    dim = 2 if Q == 9 else 3
    L = [nx, ny, nz]
    wax = dim - 1
    rng = np.random.default_rng(5)
    for i in range(Q):
        s = oracle.Sim(Q, nx, ny, nz, tau=1e30, walls=walls, wetting=False)
        f = np.broadcast_to(w.reshape(Q, 1, 1, 1), (Q, nz, ny, nx)).copy()
        X = [int(rng.integers(0, L[k])) for k in range(3)]
        if dim == 2:
            X[2] = 0
        if walls:
            X[wax] = 1   # next to the lower wall
        f[i, X[2], X[1], X[0]] += 1.0
        s.set_populations(f)
        s.step(1)
        g = s.populations() - w.reshape(Q, 1, 1, 1)
        Y = [X[k] + c[i, k] for k in range(3)]
        if walls and (Y[wax] <= 0 or Y[wax] >= L[wax] - 1):
            exp_plane, Y = opp[i], X           # bounced back into the same cell
        else:
            exp_plane = i
            Y = [Y[k] % L[k] for k in range(3)]
        assert abs(g[exp_plane, Y[2], Y[1], Y[0]] - 1.0) < 1e-14
        g[exp_plane, Y[2], Y[1], Y[0]] = 0.0
        if walls:
            solid = np.zeros(g.shape[1:], bool)
            idx = [slice(None)] * 3
            idx[2 - wax] = 0
            solid[tuple(idx)] = True
            idx[2 - wax] = L[wax] - 1
            solid[tuple(idx)] = True
            g[:, solid] = 0.0
        assert np.max(np.abs(g)) < 1e-14
        s.close()


@pytest.mark.parametrize("Q,dims", [(9, (12, 10, 1)), (19, (8, 6, 7))])
def test_rest_state_is_fixed_point(Q, dims):
    s = oracle.Sim(Q, *dims, tau=0.7, walls=True, wetting=False)
    _, w, _ = oracle.lattice(Q)
    f0 = s.populations()
    s.step(25)
    # fixed point up to round-off (sum_i w_i is 1 only to the last bit)
    assert np.max(np.abs(s.populations() - f0)) < 1e-15
    assert np.array_equal(f0[:, 0, 0, 0], w)


@pytest.mark.parametrize("Q,dims", [(9, (16, 12, 1)), (19, (8, 7, 6))])
def test_periodic_conservation(Q, dims):
    c, _, _ = oracle.lattice(Q)
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    f0 = near_eq_populations(Q, shape, seed=7)
    # no force: mass and momentum conserved
    s = oracle.Sim(Q, nx, ny, nz, tau=0.8, walls=False, wetting=False)
    s.set_populations(f0)
    m0, p0 = f0.sum(), momentum(c, f0)
    s.step(40)
    f = s.populations()
    assert abs(f.sum() - m0) < 1e-12 * m0
    assert np.allclose(momentum(c, f), p0, atol=1e-13)
    s.close()
    # uniform body force: momentum grows by sum_x F per step
    g = np.array([2e-5, -1e-5, 3e-6 if Q == 19 else 0.0])
    s = oracle.Sim(Q, nx, ny, nz, tau=0.8, walls=False, wetting=False, body_force=tuple(g))
    s.set_populations(f0)
    s.step(10)
    f = s.populations()
    assert abs(f.sum() - m0) < 1e-12 * m0
    assert np.allclose(momentum(c, f), p0 + 10 * g * nx * ny * nz, atol=1e-13)
    s.close()


def test_tension_conserves_momentum_periodic_2d():
    c, _, _ = oracle.lattice(9)
    s = oracle.Sim(9, 40, 40, tau=0.9, walls=False, wetting=False, sigma=0.01)
    rng = np.random.default_rng(8)
    s.set_interface(W.circle(50, 9.0, (20.3, 19.7)) + rng.uniform(-0.4, 0.4, (50, 2)))
    f0 = s.populations()
    s.step(60)
    f = s.populations()
    assert abs(f.sum() - f0.sum()) < 1e-12 * f0.sum()
    assert np.allclose(momentum(c, f), 0.0, atol=1e-13)


def test_tension_conserves_momentum_periodic_3d():
    c, _, _ = oracle.lattice(19)
    s = oracle.Sim(19, 16, 16, 16, tau=0.9, walls=False, wetting=False, sigma=0.01)
    rng = np.random.default_rng(9)
    q, tri = W.icosphere(2, 4.5, (8.2, 7.9, 8.1))
    s.set_interface(q + rng.uniform(-0.2, 0.2, q.shape), tri)
    f0 = s.populations()
    s.step(8)
    f = s.populations()
    assert abs(f.sum() - f0.sum()) < 1e-12 * f0.sum()
    assert np.allclose(momentum(c, f), 0.0, atol=1e-13)


def poiseuille(Q, tau, H, g, steps):
    """Body-force channel flow between the halfway walls; returns (y, u_x)."""
    if Q == 9:
        s = oracle.Sim(9, 3, H + 2, tau=tau, walls=True, wetting=False, body_force=(g, 0, 0))
    else:
        s = oracle.Sim(19, 2, 3, H + 2, tau=tau, walls=True, wetting=False,
                       body_force=(g, 0, 0))
    s.step(steps)
    rho, u, _ = s.fields()
    ux = u[0, 0, :, 0] if Q == 9 else u[0, :, 0, 0]
    s.close()
    return np.arange(H + 2), ux


@pytest.mark.parametrize("Q", [9, 19])
def test_poiseuille_exact_at_magic_tau(Q):
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    H, g = 10, 1e-6
    y, ux = poiseuille(Q, tau, H, g, 25000)
    nu = (tau - 0.5) / 3.0
    ua = g / (2 * nu) * (y - 0.5) * (H + 0.5 - y)
    fl = slice(1, H + 1)
    assert np.max(np.abs(ux[fl] - ua[fl])) < 1e-9 * ua.max()


def test_poiseuille_not_exact_elsewhere():
    # at tau = 1 halfway bounce-back has the known tau-dependent slip: the
    # profile is close (second order) but measurably off
    y, ux = poiseuille(9, 1.0, 10, 1e-6, 25000)
    ua = 1e-6 / (2 * (0.5 / 3)) * (y - 0.5) * (10.5 - y)
    err = np.max(np.abs(ux[1:11] - ua[1:11])) / ua.max()
    assert 1e-4 < err < 1e-2


def test_viscosity_matches_paper_pairs():
    rows = []
    with open(os.path.join(GOLDEN, "paper_viscosity.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                rows.append((float(parts[0]), float(parts[1])))
    assert len(rows) == 3
    H, g = 20, 1e-7
    for tau, mu in rows:
        steps = int(6 * H * H / ((tau - 0.5) / 3.0))
        y, ux = poiseuille(9, tau, H, g, steps)
        # mean velocity of the parabolic profile: g H^2 / (12 nu)
        nu_meas = g * H * H / (12.0 * ux[1:H + 1].mean())
        assert abs(nu_meas / mu - 1.0) < 5e-3, (tau, nu_meas, mu)


def test_laplace_pressure_free_droplet_2d():
    R, sigma = 12.0, 0.01
    s = oracle.Sim(9, 64, 64, tau=1.0, walls=False, wetting=False, sigma=sigma)
    s.set_interface(W.circle(76, R, (32.0, 32.0)))
    s.step(3000)
    rho, u, q = s.fields()
    yy, xx = np.mgrid[0:64, 0:64]
    r = np.hypot(xx - 32.0, yy - 32.0)
    dp = (rho[0][r < R - 3].mean() - rho[0][r > R + 4].mean()) / 3.0
    Rf = np.linalg.norm(q - q.mean(0), axis=1).mean()
    assert abs(dp / (sigma / Rf) - 1.0) < 0.02
    assert np.abs(u).max() < 1e-4 * 3   # spurious currents stay small
    s.close()


def wet_drop(theta, xi, R=10.0, steps=4000, sigma=0.01, nx=72, ny=36):
    s = oracle.Sim(9, nx, ny, tau=1.0, walls=True, wetting=True, sigma=sigma, xi=xi,
                   theta_eq_deg=theta)
    N = int(round(2 * math.pi * R / 0.7))
    s.set_interface(W.circle(N, R, (nx / 2.0, 0.5 + R + 2 * xi)))
    rc = s.step(steps)
    o = s.observables()
    A = s.A
    s.close()
    return rc, o, A


def film_root(A, xi, n, m, p):
    """Root eps of Pi(eps) = p near xi (bisection on the closed form)."""
    lo, hi = 0.5 * xi, 1.0 * xi
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        val = A * ((xi / mid) ** n - (xi / mid) ** m) - p
        lo, hi = (mid, hi) if val > 0 else (lo, mid)
    return 0.5 * (lo + hi)


def test_film_thickness_scales_with_xi():
    films = []
    for xi in (0.5, 1.0, 2.0):
        rc, o, A = wet_drop(90.0, xi)
        assert rc == 0
        films.append(o["film"])
        # the film sits where the wetting pressure balances the Laplace
        # pressure of the cap: Pi(eps) = sigma / R
        eps = film_root(A, xi, 9, 3, 0.01 / o["radius"])
        assert abs(o["film"] - eps) < 0.01 * xi
    # eps -> 0 linearly as xi -> 0
    assert abs(films[1] / films[0] - 2.0) < 0.05
    assert abs(films[2] / films[1] - 2.0) < 0.05


def test_contact_angle_follows_theta_eq():
    # with the film resolved (xi = 2 lu) the fitted angle settles near theta_eq
    # (Eq. 11 as printed, film of the outer phase); the remaining excess
    # shrinks further as xi / dx grows and with time
    th = []
    for t in (60.0, 90.0, 120.0):
        rc, o, _ = wet_drop(t, 2.0, R=12.0, steps=8000, nx=80, ny=40)
        assert rc == 0
        th.append(o["theta_deg"])
    assert th[0] < th[1] < th[2]
    assert all(0.0 < m - t < 12.0 for m, t in zip(th, (60.0, 90.0, 120.0))), th


def test_drop_2d_128x64_volume_drift_and_wall():
    wl = W.drop_2d_128x64()
    s = oracle.Sim(9, wl.nx, wl.ny, tau=wl.tau, walls=True, wetting=True, sigma=wl.sigma,
                   xi=wl.xi, theta_eq_deg=wl.theta_eq_deg, pi_n=wl.pi_n, pi_m=wl.pi_m)
    s.set_interface(wl.nodes)
    v0 = s.observables()["volume"]
    assert abs(v0 / (math.pi * 20.0 ** 2) - 1) < 1e-3
    assert s.step(wl.steps) == 0
    o = s.observables()
    assert abs(o["volume"] / v0 - 1.0) < 0.01
    assert o["d_min"] > 0.0
    # mass: the walls and forcing keep total mass fixed (no sources)
    assert abs(o["mass"] / (wl.nx * (wl.ny - 2)) - 1.0) < 1e-12
    s.close()
