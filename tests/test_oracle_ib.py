"""Pins of the oracle's IB coupling (Sec. II A, eqs. force_spread,
vel_interpolation and the four-point kernel Psi): kernel identities,
brute-force spreading on tiny grids, exact reproduction of constant and linear
velocity fields, force conservation and spread/interpolation adjointness."""
import itertools
import math

import numpy as np
import pytest


def test_psi_values_and_continuity(orc):
    assert orc.psi(0.0) == 0.5
    assert orc.psi(1.0) == 0.25
    assert orc.psi(2.0) == 0.0 and orc.psi(-2.0) == 0.0 and orc.psi(2.7) == 0.0
    for r in (1.0, 2.0):
        assert abs(orc.psi(r - 1e-12) - orc.psi(r + 1e-12)) < 1e-9
    # the second branch, evaluated at r = 1, also gives 1/4
    assert math.isclose(0.625 - 0.25 - 0.25 * math.sqrt(3 - 1 - 1.75), 0.25)
    for r in np.linspace(-3, 3, 61):
        assert orc.psi(r) == orc.psi(-r) and orc.psi(r) >= 0.0


@pytest.mark.parametrize("x", [0.0, 0.13, 0.5, 0.77, 0.999])
def test_psi_moment_conditions(orc, x):
    ks = np.arange(-3, 5)
    v = np.array([orc.psi(x - k) for k in ks])
    assert math.isclose(v.sum(), 1.0, abs_tol=1e-15)                  # partition of unity
    assert abs(((x - ks) * v).sum()) < 1e-15                           # first moment
    assert math.isclose((v ** 2).sum(), 3.0 / 8.0, abs_tol=1e-15)      # sum of squares


def brute_spread(p, xyz, phi, nzf, walls):
    """Direct evaluation over every cell and every node with minimum-image
    periodic distances; cells outside the fluid are not part of the grid."""
    nx, ny = p.nx, p.ny
    F = np.zeros((3, nzf, ny, nx))
    for z, y, x in itertools.product(range(nzf), range(ny), range(nx)):
        Z = z + 1 if walls else z
        for q, f in zip(xyz, phi):
            dx = (x - q[0] + nx / 2) % nx - nx / 2
            dy = (y - q[1] + ny / 2) % ny - ny / 2
            dz = Z - q[2]
            if not walls:
                dz = (dz + p.nz / 2) % p.nz - p.nz / 2
            w = psi_ref(dx) * psi_ref(dy) * psi_ref(dz)
            F[:, z, y, x] += f * w
    return F.reshape(-1)


def psi_ref(r):
    r = abs(r)
    if r <= 1:
        return 3 / 8 - r / 4 + math.sqrt(r - r * r + 1 / 4) / 4
    if r <= 2:
        return 5 / 8 - r / 4 - math.sqrt(3 * r - r * r - 7 / 4) / 4
    return 0.0


@pytest.mark.parametrize("walls", [0, 1])
def test_spread_matches_brute_force(orc, walls):
    rng = np.random.default_rng(11 + walls)
    nx, ny, nz = 7, 6, 8
    p = orc.make_params(nx, ny, nz, walls=walls)
    # nodes near the periodic seams, near the walls and inside
    xyz = np.array([[0.2, 5.7, 1.3], [6.5, 0.1, 3.4], [3.3, 2.9, 6.2]])
    phi = rng.standard_normal((3, 3))
    nzf = nz - 2 if walls else nz
    F = orc.spread(p, xyz, phi)
    assert np.allclose(F, brute_spread(p, xyz, phi, nzf, walls), atol=1e-15)


def test_spread_conserves_total_force(orc):
    rng = np.random.default_rng(2)
    p = orc.make_params(9, 9, 9, walls=0)
    xyz = rng.uniform(0, 9, (20, 3))
    phi = rng.standard_normal((20, 3))
    F = orc.spread(p, xyz, phi).reshape(3, -1)
    assert np.allclose(F.sum(1), phi.sum(0), atol=1e-13)


def test_interp_reproduces_constant_and_linear_fields(orc):
    rng = np.random.default_rng(3)
    nx, ny, nz = 12, 11, 12
    p = orc.make_params(nx, ny, nz, walls=1)
    Z, Y, X = np.meshgrid(np.arange(1, nz - 1), np.arange(ny), np.arange(nx), indexing="ij")
    a = rng.standard_normal(3)
    B = rng.standard_normal((3, 3))
    U = np.stack([a[k] + B[k, 0] * X + B[k, 1] * Y + B[k, 2] * Z for k in range(3)]).reshape(-1)
    # nodes whose 4x4x4 support stays inside the fluid and away from the seams
    xyz = rng.uniform([2.5, 2.5, 3.0], [nx - 4.5, ny - 4.5, nz - 5.0], (10, 3))
    qd = orc.interp(p, xyz, U)
    assert np.allclose(qd, a + xyz @ B.T, atol=1e-12)


def test_interp_wall_cells_supply_zero(orc):
    """A node next to the bottom wall: the stencil layer Z = 0 is solid and
    contributes nothing (no renormalisation of the remaining weights)."""
    p = orc.make_params(8, 8, 8, walls=1)
    U = np.ones(3 * 8 * 8 * 6)
    q = np.array([[4.0, 4.0, 1.25]])
    qd = orc.interp(p, q, U)
    wz_fluid = sum(psi_ref(Z - 1.25) for Z in range(1, 4))
    assert np.allclose(qd, wz_fluid, atol=1e-15)
    assert qd[0, 0] < 1.0


def test_spread_interp_adjoint(orc):
    rng = np.random.default_rng(4)
    for walls in (0, 1):
        p = orc.make_params(10, 9, 11, walls=walls)
        nzf = 9 if walls else 11
        xyz = rng.uniform(0, 9, (15, 3))
        xyz[:, 2] = rng.uniform(0.6, 9.5, 15)
        phi = rng.standard_normal((15, 3))
        U = rng.standard_normal(3 * 10 * 9 * nzf)
        F = orc.spread(p, xyz, phi)
        qd = orc.interp(p, xyz, U)
        assert math.isclose(F @ U, (phi * qd).sum(), rel_tol=1e-12)
