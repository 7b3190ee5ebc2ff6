"""FP64 numpy oracle of the warm start's mesh geometry.

TEST INFRASTRUCTURE ONLY: imported by tests/.  Shares no code with the CUDA
library.

* profile(xyz, R0, nphi): the App. B description of a droplet surface, the
  radial distance r = G(phi) from the droplet's centre (taken, as for the
  paper's G_sim, as the centroid of the nodes), phi the polar angle from +z,
  averaged over the azimuth (eq. L2-error_equilibrium integrates over phi
  only) -- here node by node in nphi equal bins of phi; g = G / R0; a bin
  without nodes takes the linear interpolation of its nearest filled
  neighbours (the end value beyond the first or last filled bin).
* deform(g, R0, xyz, tri, cx, cy, z_bottom): the inverse map, nodes of a
  sphere-like mesh moved onto the star-shaped surface of revolution
  r = R0 g(phi) (g linear between the bin centres phi_k = (k + 1/2) pi / nphi,
  constant beyond the end ones): each node keeps its azimuth about its
  centroid and the fraction of surface area between it and the top pole
  ((1 - cos phi)/2 on the sphere; on the target, the area of the surface of
  revolution, dA = 2 pi r sin(phi) sqrt(r^2 + r'^2) dphi, integrated by the
  midpoint rule on 4096 intervals and inverted by linear interpolation);
  then rescaled to the input mesh's enclosed volume, centred at (cx, cy),
  lowest node at z_bottom.
* cap_profile(theta, nphi): g of an exact spherical cap of contact angle
  theta resting on a plane, about the centroid of its surface (cap and
  base disc), for a cap of the volume of a unit sphere; by ray casting from
  the centroid.
"""
from __future__ import annotations

import numpy as np


def mesh_volume(xyz, tri):
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    return float(np.sum(np.einsum("ij,ij->i", a, np.cross(b, c)))) / 6.0


def profile(xyz, R0, nphi=64):
    xyz = np.asarray(xyz, np.float64)
    c = xyz.mean(axis=0)
    d = xyz - c
    r = np.sqrt(np.sum(d * d, axis=1))
    keep = r > 0
    phi = np.arccos(np.clip(d[keep, 2] / r[keep], -1.0, 1.0))
    k = np.clip((phi / np.pi * nphi).astype(int), 0, nphi - 1)
    g = np.full(nphi, np.nan)
    for b in range(nphi):
        sel = k == b
        if np.any(sel):
            g[b] = np.mean(r[keep][sel]) / R0
    filled = np.flatnonzero(~np.isnan(g))
    empty = np.flatnonzero(np.isnan(g))
    if empty.size:
        g[empty] = np.interp(empty, filled, g[filled])
    return g


def profile_at(g, phi):
    nphi = len(g)
    centres = (np.arange(nphi) + 0.5) * np.pi / nphi
    return np.interp(phi, centres, g)


def surface_area_fraction(g, R0, n=4096):
    """Cumulative area of r = R0 g(phi) from the top pole at phi_i = pi i / n."""
    h = np.pi / n
    mid = (np.arange(n) + 0.5) * h
    r = R0 * profile_at(g, mid)
    dr = R0 * (profile_at(g, mid + 0.5 * h) - profile_at(g, mid - 0.5 * h)) / h
    dA = 2.0 * np.pi * r * np.sin(mid) * np.sqrt(r * r + dr * dr) * h
    return np.concatenate([[0.0], np.cumsum(dA)])


def deform(g, R0, xyz, tri, cx, cy, z_bottom):
    g = np.asarray(g, np.float64)
    xyz = np.asarray(xyz, np.float64)
    tri = np.asarray(tri)
    c = xyz.mean(axis=0)
    d = xyz - c
    r = np.sqrt(np.sum(d * d, axis=1))
    frac = 0.5 * (1.0 - np.clip(d[:, 2] / r, -1.0, 1.0))
    A = surface_area_fraction(g, R0)
    n = len(A) - 1
    phi = np.interp(frac * A[-1], A, np.pi * np.arange(n + 1) / n)
    psi = np.arctan2(d[:, 1], d[:, 0])
    G = R0 * profile_at(g, phi)
    q = np.stack([G * np.sin(phi) * np.cos(psi), G * np.sin(phi) * np.sin(psi), G * np.cos(phi)], axis=1)
    s = np.cbrt(mesh_volume(d, tri) / mesh_volume(q, tri))
    q = s * q
    out = q + np.array([cx, cy, 0.0])
    out[:, 2] += z_bottom - q[:, 2].min()
    return out


def cap_profile(theta, nphi=64):
    """Exact profile of a spherical cap (contact angle theta in radians) of
    volume 4 pi / 3 about the centroid of its boundary surface."""
    ct = np.cos(theta)
    rho = np.cbrt(4.0 / (2.0 - 3.0 * ct + ct ** 3))   # sphere radius of the cap, V = 4 pi / 3
    zc = -rho * ct                                     # sphere centre height above the plane z = 0
    a = rho * np.sin(theta)                            # base radius
    hcap = rho * (1.0 - ct)
    # centroid of the surface (spherical cap area A_s at height z_s, base disc at 0)
    A_s = 2.0 * np.pi * rho * hcap
    # area-weighted mean height of the spherical zone between z = 0 and
    # z = hcap: on a sphere, area is uniform in z (Archimedes), so it is the
    # midpoint
    z_s = 0.5 * hcap
    A_b = np.pi * a * a
    z0 = A_s * z_s / (A_s + A_b)
    phis = (np.arange(nphi) + 0.5) * np.pi / nphi
    g = np.empty(nphi)
    for i, p in enumerate(phis):
        u = np.array([np.sin(p), np.cos(p)])           # direction (radial, z) from (0, z0)
        # distance to the plane z = 0 (only for downward rays)
        t_plane = -z0 / u[1] if u[1] < 0 else np.inf
        # distance to the sphere |(0, z0) + t u - (0, zc)| = rho, largest root
        bq = u[1] * (z0 - zc)
        cq = (z0 - zc) ** 2 - rho * rho
        t_sph = -bq + np.sqrt(bq * bq - cq)
        # the ray leaves the cap through whichever boundary it meets: the
        # sphere part lies above the plane
        hit_z = z0 + t_sph * u[1]
        g[i] = t_sph if hit_z >= 0.0 else t_plane
    return g
