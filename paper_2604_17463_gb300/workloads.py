"""Seeded synthetic inputs: initial interface shapes and workload sizes.

This module holds no arithmetic of the method itself (no lattice Boltzmann,
no forces, no delta kernel): only the geometry of the initial droplet shapes
and the sizes and parameters of the droplet workloads.  Both the CUDA path and
the CPU oracle take their inputs from here.

Shapes follow the paper's workloads (Sec. 3-4): droplets of radius R_0
resolved by a closed interface (a triangulated sphere in 3D; a closed ring in
2D), placed just above a flat wall, with xi / R_0 = 0.05.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

WALL_PLANE = 0.5  # lower wall plane with the first layer solid (halfway bounce-back)
BASE_SEED = 20260417


# ------------------------------------------------------------------ 2D rings
def circle(n: int, radius: float, centre: Tuple[float, float]) -> np.ndarray:
    """n nodes on a circle, counter-clockwise, node 0 at angle 0. [n, 2]"""
    a = 2.0 * np.pi * np.arange(n) / n
    return np.stack([centre[0] + radius * np.cos(a), centre[1] + radius * np.sin(a)], axis=1)


def truncated_circle(n: int, radius: float, theta0_deg: float, base_y: float,
                     centre_x: float) -> np.ndarray:
    """Closed CCW ring: a circular arc of the given radius meeting the line
    y = base_y at the angle theta0 (measured inside the drop), closed by the
    flat base on that line.  Nodes are spread uniformly in arc length. [n, 2]"""
    th = math.radians(theta0_deg)
    yc = base_y - radius * math.cos(th)          # centre height
    half = radius * math.sin(th)                 # half chord on the base line
    arc_len = 2.0 * th * radius                  # arc above the base line
    base_len = 2.0 * half
    total = arc_len + base_len
    s = (np.arange(n) + 0.5) * total / n
    pts = np.zeros((n, 2))
    # parametrise: start at the right end of the base, walk the arc CCW to the
    # left end, then walk the base back left -> right.
    a_start = math.pi / 2 - th                   # angle of the right contact point
    for k, sk in enumerate(s):
        if sk < arc_len:
            ang = a_start + sk / radius
            pts[k] = (centre_x + radius * math.cos(ang), yc + radius * math.sin(ang))
        else:
            t = sk - arc_len
            pts[k] = (centre_x - half + t, base_y)
    return pts


# ------------------------------------------------------------------ 3D mesh
def icosphere(level: int, radius: float, centre: Tuple[float, float, float]):
    """Icosahedron refined `level` times by 1 -> 4 midpoint subdivision with
    every vertex projected to the sphere.  Faces are oriented outward.
    Returns (nodes [10*4^level + 2, 3], faces [20*4^level, 3] int32)."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v += [(0.0, s1, s2 * g), (s1, s2 * g, 0.0), (s2 * g, 0.0, s1)]
    verts = np.array(v)
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    # faces: triples of mutually adjacent vertices (edge = minimum distance)
    d = np.linalg.norm(verts[:, None, :] - verts[None, :, :], axis=2)
    edge = np.min(d[d > 1e-9])
    adj = np.abs(d - edge) < 1e-6
    faces = []
    for a in range(12):
        for b in range(a + 1, 12):
            if not adj[a, b]:
                continue
            for c in range(b + 1, 12):
                if adj[a, c] and adj[b, c]:
                    n = np.cross(verts[b] - verts[a], verts[c] - verts[a])
                    if np.dot(n, verts[a] + verts[b] + verts[c]) < 0:
                        faces.append((a, c, b))
                    else:
                        faces.append((a, b, c))
    verts = [tuple(x) for x in verts]
    for _ in range(level):
        cache = {}
        new_faces = []

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                p = np.add(verts[i], verts[j]) * 0.5
                p /= np.linalg.norm(p)
                cache[key] = len(verts)
                verts.append(tuple(p))
            return cache[key]

        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    nodes = np.asarray(verts) * radius + np.asarray(centre)[None, :]
    return nodes, np.asarray(faces, dtype=np.int32)


def icosphere_level_for(radius: float, max_edge: float = 1.5) -> int:
    """Smallest subdivision level whose mean edge is at most max_edge lu."""
    for lvl in range(0, 8):
        nodes, faces = icosphere(lvl, radius, (0.0, 0.0, 0.0))
        e = np.linalg.norm(nodes[faces[:, 0]] - nodes[faces[:, 1]], axis=1).mean()
        if e <= max_edge:
            return lvl
    return 7


# ------------------------------------------------------------------ workloads
@dataclasses.dataclass
class Workload:
    """One droplet simulation: lattice, physical parameters, initial interface."""
    name: str
    lattice: int                 # 9 or 19
    nx: int
    ny: int
    nz: int
    tau: float
    sigma: float
    xi: float
    theta_eq_deg: float
    pi_n: int
    pi_m: int
    steps: int
    nodes: np.ndarray            # [N, dim]
    faces: Optional[np.ndarray]  # [M, 3] (3D) or None
    walls: bool = True
    wetting: bool = True

    @property
    def dim(self) -> int:
        return 2 if self.lattice == 9 else 3

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def fluid_cells(self) -> int:
        if not self.walls:
            return self.cells
        if self.dim == 2:
            return self.nx * (self.ny - 2)
        return self.nx * self.ny * (self.nz - 2)


def drop_2d_128x64() -> Workload:
    """2D D2Q9 128x64, tau = 1, circle R = 20 with 200 nodes centred 22 lu
    above the wall, sigma = 1e-3, theta_eq = 60 deg, xi = 0.05 R, 2000 steps."""
    R = 20.0
    nodes = circle(200, R, (64.0, WALL_PLANE + 22.0))
    return Workload("d2q9_128x64_fp64", 9, 128, 64, 1, 1.0, 1e-3, 0.05 * R, 60.0, 9, 3,
                    2000, nodes, None)


def spreading_2d_2048x512(theta_eq_deg: float = 60.0, tau: float = 1.0, downscale: int = 1) -> Workload:
    """2D D2Q9 2048x512 spreading, R = 200 with 2000 nodes, initial angle
    150 deg; optional downscaled copy (lattice, R, nodes / downscale)."""
    R = 200.0 / downscale
    xi = 0.05 * R
    n = 2000 // downscale
    nx, ny = 2048 // downscale, 512 // downscale
    nodes = truncated_circle(n, R, 150.0, WALL_PLANE + xi, nx / 2.0)
    return Workload(f"d2q9_spread_{nx}x{ny}", 9, nx, ny, 1, tau, 1e-3, xi, theta_eq_deg, 9, 3,
                    200000, nodes, None)


def drop_3d_256x256x128() -> Workload:
    """3D D3Q19 256x256x128, icosphere R = 40 (20480 faces, 10242 nodes)
    centred 42 lu above the wall, theta_eq = 75 deg, tau = 0.8."""
    R = 40.0
    nodes, faces = icosphere(5, R, (128.0, 128.0, WALL_PLANE + 42.0))
    return Workload("d3q19_256x256x128", 19, 256, 256, 128, 0.8, 1e-3, 0.05 * R, 75.0, 9, 3,
                    50000, nodes, faces)


def droplet_2d(width: int, theta_eq_deg: float, tau: float, steps: int,
               name: str = "d2q9") -> Workload:
    """Batched / served 2D member: height = width / 4, R = height / 3,
    10 nodes per unit radius, xi = max(0.05 R, 1 lu); the lowest node starts
    at the film distance xi from the wall (as the paper's drop placed at
    d ~ eps from the wall, Sec. 4)."""
    ny = max(width // 4, 12)
    R = ny / 3.0
    xi = max(0.05 * R, 1.0)
    n = int(round(10 * R))
    nodes = circle(n, R, (width / 2.0, WALL_PLANE + R + xi))
    return Workload(f"{name}_{width}x{ny}", 9, width, ny, 1, tau, 1e-3, xi, theta_eq_deg, 9, 3,
                    steps, nodes, None)


def droplet_3d(nx: int, ny: int, nz: int, theta_eq_deg: float, tau: float, steps: int,
               name: str = "d3q19") -> Workload:
    """Served 3D member: R = nz / 3, icosphere refined to mean edge <= 1.5 lu,
    lowest node at the film distance xi from the wall."""
    R = nz / 3.0
    xi = max(0.05 * R, 1.0)
    lvl = icosphere_level_for(R)
    nodes, faces = icosphere(lvl, R, (nx / 2.0, ny / 2.0, WALL_PLANE + R + xi))
    return Workload(f"{name}_{nx}x{ny}x{nz}", 19, nx, ny, nz, tau, 1e-3, xi, theta_eq_deg, 9, 3,
                    steps, nodes, faces)


def batch_2d_drops(count: int = 256, seed: int = BASE_SEED + 4, steps_lo: int = 5000,
            steps_hi: int = 50000) -> List[Workload]:
    """256 uneven 2D droplets: width log-uniform in [64, 1024], theta_eq
    uniform in [30, 150], tau uniform in [0.55, 1.5]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        w = int(round(math.exp(rng.uniform(math.log(64), math.log(1024)))))
        th = float(rng.uniform(30.0, 150.0))
        tau = float(rng.uniform(0.55, 1.5))
        st = int(rng.integers(steps_lo, steps_hi + 1))
        out.append(droplet_2d(w, th, tau, st, name=f"drop{k:03d}"))
    return out


@dataclasses.dataclass
class Request:
    arrival_s: float
    work: Workload


def serve_requests(count: int = 2000, rate_per_s: float = 50.0, seed: int = BASE_SEED + 5,
            steps_lo: int = 5000, steps_hi: int = 50000, frac_3d: float = 0.2) -> List[Request]:
    """Poisson stream of wetting requests: 80% 2D (sizes as in the batched
    workload), 20% 3D D3Q19 between 64^3 and 192x192x96."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        th = float(rng.uniform(30.0, 150.0))
        tau = float(rng.uniform(0.55, 1.5))
        st = int(rng.integers(steps_lo, steps_hi + 1))
        if rng.uniform() < frac_3d:
            s = float(rng.uniform(0.0, 1.0))
            nx = int(round(64 + s * (192 - 64)))
            nz = int(round(64 + s * (96 - 64)))
            out.append(Request(t, droplet_3d(nx, nx, nz, th, tau, st, name=f"req{k:04d}")))
        else:
            w = int(round(math.exp(rng.uniform(math.log(64), math.log(1024)))))
            out.append(Request(t, droplet_2d(w, th, tau, st, name=f"req{k:04d}")))
    return out


# ------------------------------------------------------------------ random data
def random_perturbation(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded uniform noise in [-scale, scale]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=shape)


# --------------------------------------------------------- drop in shear flow
@dataclasses.dataclass
class ShearDrop:
    """A free drop at the centre of a wall-bounded shear flow (Sec. 4): walls
    at z = 1/2 and z = nz - 3/2 (y in 2D) moving at -/+ gamma_dot H / 2 along
    x, the fluid initially in the fully developed linear profile.  Re and Ca
    use the outer (matrix) viscosity mu = (tau_out - 1/2) / 3 and rho = 1:
    Re = gamma_dot R0^2 / nu, Ca = mu gamma_dot R0 / sigma; the viscosity
    ratio is lambda = (tau - 1/2) / (tau_out - 1/2)."""
    work: Workload
    gamma_dot: float
    tau_out: float
    Re: float
    Ca: float
    R0: float

    @property
    def lam(self) -> float:
        return (self.work.tau - 0.5) / (self.tau_out - 0.5)

    @property
    def height(self) -> float:
        wl = self.work
        return float((wl.ny if wl.dim == 2 else wl.nz) - 2)

    @property
    def wall_u_lo(self):
        return (-0.5 * self.gamma_dot * self.height, 0.0, 0.0)

    @property
    def wall_u_hi(self):
        return (0.5 * self.gamma_dot * self.height, 0.0, 0.0)

    @property
    def t_mu(self) -> float:
        """Capillary time mu R0 / sigma = Ca / gamma_dot (steps)."""
        return self.Ca / self.gamma_dot

    def d_inf(self) -> float:
        """Small-deformation steady deformation of an unbounded 3D drop
        (Sec. 4, Eq. 16): (19 lambda + 16) / (16 lambda + 16) Ca."""
        lam = self.lam
        return (19.0 * lam + 16.0) / (16.0 * lam + 16.0) * self.Ca

    def initial_velocity(self) -> np.ndarray:
        """Linear shear profile u_x = gamma_dot (a - a_c) on the fluid layers
        (zero in the solid layers), [dim][nz][ny][nx]."""
        wl = self.work
        u = np.zeros((wl.dim, wl.nz, wl.ny, wl.nx))
        La = wl.ny if wl.dim == 2 else wl.nz
        ac = 0.5 + 0.5 * self.height
        prof = self.gamma_dot * (np.arange(La) - ac)
        prof[0] = prof[-1] = 0.0
        if wl.dim == 2:
            u[0] = prof[None, :, None]
        else:
            u[0] = prof[:, None, None]
        return u


def shear_drop(R0: float = 19.0, Re: float = 0.01, Ca: float = 0.05, tau: float = 1.0,
               tau_out: Optional[float] = None, nx: int = 160, ny: int = 128, nz: int = 242,
               level: Optional[int] = None, t_mu_count: float = 12.0,
               lattice: int = 19) -> ShearDrop:
    """The drop-in-shear case of Sec. 4 (defaults: Re = 0.01, Ca = 0.05,
    R0 = 19, tau = 1, lambda = 1) in a channel of nz - 2 fluid layers.  The
    drop centre is offset by a fraction of a lattice spacing from the
    lattice's symmetry planes.  Steps: t_mu_count capillary times."""
    tau_out = tau if tau_out is None else tau_out
    nu = (tau_out - 0.5) / 3.0
    gamma_dot = Re * nu / (R0 * R0)
    sigma = nu * gamma_dot * R0 / Ca
    if lattice == 19:
        lvl = icosphere_level_for(R0, 0.8) if level is None else level
        nodes, faces = icosphere(lvl, R0, (nx / 2.0 + 0.13, ny / 2.0 - 0.21, 0.5 + 0.5 * (nz - 2) + 0.07))
    else:
        n = int(round(2 * math.pi * R0 / 0.7))
        nodes = circle(n, R0, (nx / 2.0 + 0.13, 0.5 + 0.5 * (ny - 2) + 0.07))
        faces = None
        nz = 1
    steps = int(round(t_mu_count * Ca / gamma_dot))
    wl = Workload(f"shear_drop_R{R0:g}_Ca{Ca:g}_Re{Re:g}", lattice, nx, ny, nz, tau, sigma,
                  0.05 * R0, 90.0, 9, 3, steps, nodes, faces, walls=True, wetting=False)
    return ShearDrop(wl, gamma_dot, tau_out, Re, Ca, R0)


# ------------------------------------------------- paper-scale 3D spreading
def _icosahedron():
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v += [(0.0, s1, s2 * g), (s1, s2 * g, 0.0), (s2 * g, 0.0, s1)]
    verts = np.array(v)
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    d = np.linalg.norm(verts[:, None, :] - verts[None, :, :], axis=2)
    edge = np.min(d[d > 1e-9])
    adj = np.abs(d - edge) < 1e-6
    faces = []
    for a in range(12):
        for b in range(a + 1, 12):
            if not adj[a, b]:
                continue
            for c in range(b + 1, 12):
                if adj[a, c] and adj[b, c]:
                    n = np.cross(verts[b] - verts[a], verts[c] - verts[a])
                    faces.append((a, c, b) if np.dot(n, verts[a] + verts[b] + verts[c]) < 0
                                 else (a, b, c))
    return verts, faces


def geodesic_sphere(freq: int, radius: float, centre: Tuple[float, float, float]):
    """Class-I geodesic sphere: every icosahedron face cut into freq^2
    triangles on a barycentric grid, points projected to the sphere.  Shared
    edge and corner points are merged exactly (keyed by their integer
    barycentric combination of icosahedron vertices).  Faces outward.
    Returns (nodes [10 freq^2 + 2, 3], faces [20 freq^2, 3] int32)."""
    verts, ico = _icosahedron()
    index = {}
    pts = []

    def node(combo):
        key = tuple(sorted((v, w) for v, w in combo if w > 0))
        k = index.get(key)
        if k is None:
            p = sum(w * verts[v] for v, w in key) / freq
            k = index[key] = len(pts)
            pts.append(p / np.linalg.norm(p))
        return k

    faces = []
    for a, b, c in ico:
        grid = {}
        for i in range(freq + 1):
            for j in range(freq + 1 - i):
                grid[(i, j)] = node(((a, freq - i - j), (b, i), (c, j)))
        for i in range(freq):
            for j in range(freq - i):
                faces.append((grid[(i, j)], grid[(i + 1, j)], grid[(i, j + 1)]))
                if i + j < freq - 1:
                    faces.append((grid[(i + 1, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]))
    nodes = np.asarray(pts) * radius + np.asarray(centre)[None, :]
    return nodes, np.asarray(faces, dtype=np.int32)


def truncated_sphere(freq: int, radius: float, theta0_deg: float, base_z: float,
                     centre_xy: Tuple[float, float]):
    """Closed mesh of a spherical cap of radius `radius` meeting the plane
    z = base_z at the angle theta0 (a drop resting on its film), from the
    geodesic sphere: a point at polar angle beta from the top pole goes to
    the cap at polar angle beta theta0 / (pi/2) for beta <= pi/2, and to the
    flat base disc at radius R sin(theta0) (pi - beta) / (pi/2) below the
    equator.  Topology and outward orientation are those of the sphere."""
    unit, faces = geodesic_sphere(freq, 1.0, (0.0, 0.0, 0.0))
    th0 = math.radians(theta0_deg)
    beta = np.arccos(np.clip(unit[:, 2], -1.0, 1.0))
    phi = np.arctan2(unit[:, 1], unit[:, 0])
    zc = base_z - radius * math.cos(th0)          # sphere centre height
    out = np.zeros_like(unit)
    up = beta <= 0.5 * math.pi
    b = beta[up] * th0 / (0.5 * math.pi)
    out[up, 0] = radius * np.sin(b) * np.cos(phi[up])
    out[up, 1] = radius * np.sin(b) * np.sin(phi[up])
    out[up, 2] = zc + radius * np.cos(b)
    r = radius * math.sin(th0) * (math.pi - beta[~up]) / (0.5 * math.pi)
    out[~up, 0] = r * np.cos(phi[~up])
    out[~up, 1] = r * np.sin(phi[~up])
    out[~up, 2] = base_z
    out[:, 0] += centre_xy[0]
    out[:, 1] += centre_xy[1]
    return out, faces


@dataclasses.dataclass
class Spread3D:
    """A paper-scale 3D spreading run (Sec. 3 and 4) with its capillary time
    t_mu = mu_in R0 / sigma and the Reynolds number rho sigma R0 / mu_in^2."""
    work: Workload
    R0: float
    t_mu: float
    Re: float
    t_mu_count: float


def spread3d_cap(tau: float, R0: float = 50.0 / 2.0 ** (1.0 / 3.0), sigma: float = 1e-3,
                 freq: int = 77, t_mu_count: float = 50.0) -> Spread3D:
    """Sec. 3: 250 x 250 x 150 lattice, a drop resting as a hemisphere
    (contact angle 90 deg) on its film spreads towards theta_eq = 60 deg.
    R0 is the radius of the sphere of the same volume (the paper's reference
    radius), so the hemisphere has radius 2^(1/3) R0 (50 lu by default);
    xi / R0 = 0.05; about 120 000 triangles (20 freq^2 = 118 580 at freq 77);
    run t_mu_count capillary times t_mu = mu R0 / sigma."""
    xi = 0.05 * R0
    Rh = 2.0 ** (1.0 / 3.0) * R0
    nodes, faces = truncated_sphere(freq, Rh, 90.0, WALL_PLANE + xi, (125.0 + 0.17, 125.0 - 0.11))
    mu = (tau - 0.5) / 3.0
    t_mu = mu * R0 / sigma
    steps = int(round(t_mu_count * t_mu))
    wl = Workload(f"spread3d_cap_250x250x150_tau{tau:g}", 19, 250, 250, 150, tau, sigma, xi,
                  60.0, 9, 3, steps, nodes, faces)
    return Spread3D(wl, R0, t_mu, sigma * R0 / mu ** 2, t_mu_count)


def spread3d_sphere(R0: float = 50.0 / 2.0 ** (1.0 / 3.0), sigma: float = 1e-3, tau: float = 0.56,
                    freq: int = 77, t_mu_count: float = 50.0) -> Spread3D:
    """Sec. 4: 300 x 300 x 250 lattice, a sphere of radius R0 (the same
    reference radius as the Sec. 3 runs) whose lowest node sits at the film
    distance xi from the wall, theta_eq = 45 deg, tau = 0.56 (mu_in = 0.02),
    xi / R0 = 0.05, about 120 000 triangles."""
    xi = 0.05 * R0
    nodes, faces = geodesic_sphere(freq, R0, (150.0 + 0.17, 150.0 - 0.11, WALL_PLANE + xi + R0))
    mu = (tau - 0.5) / 3.0
    t_mu = mu * R0 / sigma
    steps = int(round(t_mu_count * t_mu))
    wl = Workload("spread3d_sphere_300x300x250", 19, 300, 300, 250, tau, sigma, xi, 45.0, 9, 3,
                  steps, nodes, faces)
    return Spread3D(wl, R0, t_mu, sigma * R0 / mu ** 2, t_mu_count)
