"""Seeded synthetic inputs: droplet meshes, workloads and perturbations.

This module holds none of the IB-LB arithmetic; it only builds inputs
(triangulated spheres, droplet placements, random perturbations).  Both the
CUDA path and the CPU oracle are fed from here by the tests and the benchmark,
which is the only thing the two sides share.

The paper (Sec. III A) starts every run from a spherical droplet of radius R0
modelled with a closed triangular mesh placed near the substrate.  The mesh
generator of the paper is not given (its N_t = 20 000 / 40 000 are not
subdivision counts); the icosphere used here gives 20 * 4**L faces and
10 * 4**L + 2 nodes (L = 3: 642 / 1280, L = 5: 10 242 / 20 480,
L = 6: 40 962 / 81 920).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def icosahedron():
    """12 vertices (two poles on the z axis) and 20 outward CCW faces."""
    v = [(0.0, 0.0, 1.0)]
    zr, rr = 1.0 / math.sqrt(5.0), 2.0 / math.sqrt(5.0)
    for k in range(5):
        a = 2.0 * math.pi * k / 5.0
        v.append((rr * math.cos(a), rr * math.sin(a), zr))
    for k in range(5):
        a = 2.0 * math.pi * k / 5.0 + math.pi / 5.0
        v.append((rr * math.cos(a), rr * math.sin(a), -zr))
    v.append((0.0, 0.0, -1.0))
    f = []
    for k in range(5):
        u0, u1 = 1 + k, 1 + (k + 1) % 5
        l0, l1 = 6 + k, 6 + (k + 1) % 5
        f.append((0, u0, u1))          # top cap
        f.append((u0, l0, u1))         # upper band
        f.append((u1, l0, l1))         # lower band
        f.append((l0, 11, l1))         # bottom cap
    return np.array(v, dtype=np.float64), np.array(f, dtype=np.int32)


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Unit icosahedron subdivided `level` times (midpoints pushed to the
    sphere), scaled by `radius` and moved to `center`.  Node order is fixed:
    the 12 icosahedron corners, then midpoints in order of creation.
    Returns (xyz float64 [N,3], tri int32 [Nt,3]) with faces CCW seen from
    outside."""
    v, f = icosahedron()
    verts = [tuple(p) for p in v]
    faces = [tuple(t) for t in f]
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                p = np.add(verts[a], verts[b])
                p = p / np.linalg.norm(p)
                mid[key] = len(verts)
                verts.append(tuple(p))
            return mid[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    xyz = np.array(verts, dtype=np.float64) * radius + np.asarray(center, dtype=np.float64)
    return xyz, np.array(faces, dtype=np.int32)


def level_for_radius(R: float) -> int:
    """Icosphere level for a droplet of radius R (mean edge <~ 1.2 lattice
    units): L3 below R = 9, L4 below R = 17, else L5."""
    if R < 9:
        return 3
    if R < 17:
        return 4
    return 5


def droplet_center(nx, ny, R, xi, z_wall=0.5, gap=None):
    """Centre of a droplet whose lowest node sits a height `gap` above the
    wall plane (default gap = xi, where the wall interaction vanishes)."""
    g = xi if gap is None else gap
    return (nx / 2.0, ny / 2.0, z_wall + R + g)


def rest_populations(cells: int, w, rho0=1.0):
    """f_i = w_i rho0 on every cell, layout [i][cell]."""
    return np.repeat(np.asarray(w, np.float64)[:, None] * rho0, cells, axis=1).reshape(-1)


def perturbed_populations(cells: int, w, seed: int, amp=1e-3, rho0=1.0):
    """f_i = w_i rho0 (1 + amp * U(-1, 1)): a seeded non-equilibrium state."""
    rng = np.random.default_rng(seed)
    f = np.asarray(w, np.float64)[:, None] * rho0 * (1.0 + amp * rng.uniform(-1, 1, (19, cells)))
    return f.reshape(-1)


def jitter_nodes(xyz, seed: int, amp: float):
    """Node positions moved by a seeded uniform jitter of size `amp`."""
    rng = np.random.default_rng(seed)
    return xyz + amp * rng.uniform(-1.0, 1.0, xyz.shape)


@dataclass
class DropletSpec:
    """One droplet workload: box, fluid and membrane parameters."""
    nx: int
    ny: int
    nz: int
    R: float
    level: int
    sigma: float
    theta_deg: float
    xi: float
    tau: float = 1.0
    lam: float = 1.0
    storage: str = "f32"
    volume_correction: bool = True
    gap: float | None = None
    walls: bool = True
    extra: dict = field(default_factory=dict)

    def mesh(self):
        c = droplet_center(self.nx, self.ny, self.R, self.xi, gap=self.gap)
        return icosphere(self.level, self.R, c)

    @property
    def tau_in(self):
        # lambda = mu_in / mu_out with mu = rho cs^2 (tau - 1/2) (eq. def_lambda)
        return 0.5 + self.lam * (self.tau - 0.5)


def workload_parity_32():
    """32^3 box, walls at Z = 0 and Z = 31, tau = 1, L3 icosphere (642 nodes),
    R = 8, sigma = 0.01, theta_eq = 90 deg, xi = 2, lowest node at h = xi."""
    return DropletSpec(32, 32, 32, 8.0, 3, 0.01, 90.0, 2.0, tau=1.0, volume_correction=False)


def workload_statics_128(theta_deg=90.0, storage="f16"):
    """128^3 box, tau = 1, L5 icosphere (10 242 nodes), R = 24, sigma = 0.005,
    xi = 0.1 R = 2.4, volume correction on."""
    return DropletSpec(128, 128, 128, 24.0, 5, 0.005, theta_deg, 2.4, tau=1.0, storage=storage)


def workload_statics_64(theta_deg=90.0, storage="f32"):
    """Half-scale statics case: 64^3, R = 12, L4 mesh, xi = 2 (0.1 R = 1.2
    would fall below two lattice units)."""
    return DropletSpec(64, 64, 64, 12.0, 4, 0.005, theta_deg, 2.0, tau=1.0, storage=storage)


def workload_spreading_256(storage="bf16"):
    """256 x 256 x 128 box, tau_out = 0.8, lambda = 10, L6 icosphere (40 962
    nodes), R = 40, theta_eq = 20 deg, sigma = 0.005, xi = 2."""
    return DropletSpec(256, 256, 128, 40.0, 6, 0.005, 20.0, 2.0, tau=0.8, lam=10.0, storage=storage)


def workload_batch(n=64, seed=2025, storage="f16"):
    """n independent droplets: cubic boxes of side U{48..96}, R ~ U[6, 20],
    theta_eq ~ U[20, 160] deg, tau ~ U[0.6, 1.2], sigma = 0.01, xi =
    max(2, 0.1 R), icosphere level by radius.  numpy PCG64 with `seed`."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        s = int(rng.integers(48, 97))
        R = float(rng.uniform(6.0, 20.0))
        th = float(rng.uniform(20.0, 160.0))
        tau = float(rng.uniform(0.6, 1.2))
        xi = max(2.0, 0.1 * R)
        out.append(DropletSpec(s, s, s, R, level_for_radius(R), 0.01, th, xi, tau=tau, storage=storage))
    return out


# ----------------------------------------------------------- learned warm start
MLP_SIZES = (3, 256, 256, 256, 64)


def mlp_init(seed=0, sizes=MLP_SIZES):
    """Seeded initial parameters of the warm-start network as one float32
    vector, layer by layer W_l (out x in, row major) then b_l: weights
    uniform in +-1/sqrt(in), hidden biases 0, output biases 1 (the sphere,
    g = 1)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (i, o) in enumerate(zip(sizes[:-1], sizes[1:])):
        lim = 1.0 / np.sqrt(i)
        parts.append(rng.uniform(-lim, lim, o * i))
        parts.append(np.ones(o) if l == len(sizes) - 2 else np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def warmstart_cases(n, seed):
    """n cases (theta_eq deg, R0, lambda): theta_eq ~ U[20, 160], R0 ~ U[8, 24],
    lambda log-uniform in [0.1, 10]; numpy PCG64 with `seed`."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(20.0, 160.0, n)
    R = rng.uniform(8.0, 24.0, n)
    lam = 10.0 ** rng.uniform(-1.0, 1.0, n)
    return np.stack([th, R, lam], axis=1)
