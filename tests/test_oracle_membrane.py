"""Pins of the oracle's membrane forces: surface tension (Sec. II B) and the
wall interaction (Sec. II C, eqs. disjoin-p and A_choice, App. A)."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize

from paper_2503_20605_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden_constants():
    out = {}
    for line in open(os.path.join(GOLD, "paper_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, val = line.split()[:2]
        out[name] = val
    return out


def area_np(xyz, tri):
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum()


def jittered_sphere(level=2, R=5.0, seed=0, amp=0.3):
    xyz, tri = I.icosphere(level, R, (10.0, 11.0, 12.0))
    return I.jitter_nodes(xyz, seed, amp), tri


def params(orc, **kw):
    d = dict(sigma=0.02, wetting=0)
    d.update(kw)
    return orc.make_params(32, 32, 32, **d)


def test_surface_tension_invariants(orc):
    xyz, tri = jittered_sphere()
    sigma = 0.02
    phi, fs, fp, _ = orc.membrane_forces(params(orc, sigma=sigma), xyz, tri)
    assert np.allclose(phi, fs) and not fp.any()
    assert np.allclose(fs.sum(0), 0.0, atol=1e-14)                     # translation
    assert np.allclose(np.cross(xyz, fs).sum(0), 0.0, atol=1e-12)       # rotation
    # Euler: the area is homogeneous of degree 2 in q, so sum q.dA/dq = 2A
    assert math.isclose((xyz * fs).sum(), -2.0 * sigma * area_np(xyz, tri), rel_tol=1e-12)


def test_surface_tension_is_minus_sigma_grad_area(orc):
    xyz, tri = jittered_sphere(level=1, seed=3)
    sigma = 0.7
    _, fs, _, _ = orc.membrane_forces(params(orc, sigma=sigma), xyz, tri)
    # central differences: truncation ~h^2, rounding ~eps*A/h ~ 1e-9 here
    h = 1e-5
    for j in (0, 5, 17, len(xyz) - 1):
        for a in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[j, a] += h
            xm[j, a] -= h
            fd = -sigma * (area_np(xp, tri) - area_np(xm, tri)) / (2 * h)
            assert abs(fd - fs[j, a]) < 5e-8 * max(1.0, abs(fs[j, a]))


def fem_triangle_energy(X0, X, sigma):
    """Energy of one triangle following Sec. II B literally: linear shape
    functions N_k on the reference triangle (local 2D frame), displacement
    gradient grad V, surface deformation tensor D = I + grad V (expressed
    between the reference and the current tangent planes), invariant
    a = 1/2 log{1/2 [tr(D D^T)]^2 - 1/2 tr[(D D^T)^2]}, w(a) = sigma e^a,
    integrated over the reference area."""
    def frame(P):
        e1 = P[1] - P[0]
        n = np.cross(e1, P[2] - P[0])
        e1 = e1 / np.linalg.norm(e1)
        e2 = np.cross(n / np.linalg.norm(n), e1)
        return np.array([[(p - P[0]) @ e1, (p - P[0]) @ e2] for p in P])
    x0, x = frame(X0), frame(X)
    # shape-function gradients on the reference triangle: N_k = a_k x + b_k y + c_k
    M = np.column_stack([x0, np.ones(3)])
    coef = np.linalg.inv(M)           # columns: coefficients (a_k, b_k, c_k) of N_k
    grad_N = coef[:2, :]              # 2 x 3
    V = x - x0                        # in-plane displacements of the corners
    gradV = V.T @ grad_N.T            # dV_i / dX_j
    D = np.eye(2) + gradV
    Mdd = D @ D.T
    a = 0.5 * math.log(0.5 * np.trace(Mdd) ** 2 - 0.5 * np.trace(Mdd @ Mdd))
    w = sigma * math.exp(a)
    A0 = 0.5 * abs(np.linalg.det(np.column_stack([x0[1] - x0[0], x0[2] - x0[0]])))
    return A0 * w


def test_fem_energy_reading_equals_sigma_area(orc):
    """The reading that w is per unit reference area makes the FEM energy of
    each triangle exactly sigma times its current area, whatever the
    reference shape; the oracle's force is the gradient of that energy."""
    rng = np.random.default_rng(7)
    sigma = 0.3
    for _ in range(20):
        X0 = rng.standard_normal((3, 3))
        X = X0 + 0.4 * rng.standard_normal((3, 3))
        A = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
        assert math.isclose(fem_triangle_energy(X0, X, sigma), sigma * A, rel_tol=1e-10)
    # and its derivative equals the oracle's nodal force for a whole mesh
    xyz0, tri = I.icosphere(1, 3.0, (8.0, 8.0, 8.0))
    xyz = I.jitter_nodes(xyz0, 1, 0.2)
    _, fs, _, _ = orc.membrane_forces(params(orc, sigma=sigma), xyz, tri)
    h = 1e-6

    def energy(q):
        return sum(fem_triangle_energy(xyz0[t], q[t], sigma) for t in tri)
    for j, a in ((0, 2), (9, 0), (30, 1)):
        xp, xm = xyz.copy(), xyz.copy()
        xp[j, a] += h
        xm[j, a] -= h
        assert abs(-(energy(xp) - energy(xm)) / (2 * h) - fs[j, a]) < 1e-7


def test_surface_tension_on_sphere_is_laplace_like(orc):
    """On a fine sphere the nodal force approximates sigma (2/R) times the
    node's area share, directed inward (F_sigma = -sigma n div n)."""
    R, sigma = 10.0, 0.01
    xyz, tri = I.icosphere(4, R, (0.0, 0.0, 0.0))
    _, fs, _, _ = orc.membrane_forces(params(orc, sigma=sigma), xyz, tri)
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    At = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    chi = np.zeros(len(xyz))
    for k in range(3):
        np.add.at(chi, tri[:, k], At)
    nr = xyz / np.linalg.norm(xyz, axis=1, keepdims=True)
    radial = (fs * nr).sum(1)
    want = -sigma * 2.0 / R * chi / 3.0
    assert np.all(radial < 0)
    rel = np.abs(radial / want - 1)
    # the 12 five-valent corners of the icosahedron deviate most (the 1/3
    # area share is not their Voronoi area); everywhere else it is O(edge^2)
    assert np.median(rel) < 0.01 and rel.max() < 0.2
    assert np.sort(rel)[-13] < 0.05
    # all nodes at radius R: sum_j q_j.phi_j / R = -2 sigma A / R exactly (Euler)
    assert math.isclose(radial.sum(), -2.0 * sigma * area_np(xyz, tri) / R, rel_tol=1e-12)


def test_wetting_constants(orc):
    g = golden_constants()
    n, m = int(g["wall_exponent_n"]), int(g["wall_exponent_m"])
    sigma, xi = 0.01, 2.0
    # (m-1)(n-1)/(n-m) = 10/3 for (6, 3), with (1 + cos theta) = 1 at 90 deg
    assert math.isclose(orc.wetting_A(sigma, math.pi / 2, xi, n, m) * xi / sigma, 10.0 / 3.0)
    assert orc.wetting_A(sigma, math.pi, xi, n, m) == pytest.approx(0.0, abs=1e-18)
    A = orc.wetting_A(sigma, math.radians(40), xi, n, m)
    assert orc.Pi(xi, A, xi, n, m) == 0.0
    # minimum of Pi at h* = xi (n/m)^(1/(n-m)) = 2^(1/3) xi
    res = optimize.minimize_scalar(lambda h: orc.Pi(h, A, xi, n, m), bounds=(xi, 3 * xi),
                                   method="bounded", options={"xatol": 1e-10})
    assert math.isclose(res.x / xi, 2.0 ** (1.0 / 3.0), rel_tol=1e-6)
    assert orc.Pi(0.5 * xi, A, xi, n, m) > 0 > orc.Pi(1.5 * xi, A, xi, n, m)


@pytest.mark.parametrize("theta_deg", [20, 45, 90, 135, 160])
def test_A_choice_from_wedge_integrals(orc, theta_deg):
    """App. A: sigma int_0^(pi-theta) sin psi dpsi = -A int_xi^inf Pi(h)/A dh."""
    n, m, sigma, xi = 6, 3, 0.01, 2.0
    th = math.radians(theta_deg)
    A = orc.wetting_A(sigma, th, xi, n, m)
    lhs = sigma * integrate.quad(math.sin, 0.0, math.pi - th)[0]
    rhs = -integrate.quad(lambda h: orc.Pi(h, A, xi, n, m), xi, np.inf, epsabs=1e-14)[0]
    assert math.isclose(lhs, rhs, rel_tol=1e-8)


def test_wetting_force_direction_and_area_share(orc):
    R, xi, sigma = 6.0, 2.0, 0.01
    xyz, tri = I.icosphere(3, R, (16.0, 16.0, 0.5 + R + 0.7 * xi))   # bottom pole at h = 0.7 xi
    A = orc.wetting_A(sigma, math.radians(60), xi)
    p = params(orc, sigma=sigma, wetting=1, A=A, xi=xi)
    phi, fs, fp, clamped = orc.membrane_forces(p, xyz, tri)
    assert clamped == 0
    assert np.allclose(phi, fs + fp)
    south = int(np.argmin(xyz[:, 2]))
    h = xyz[south, 2] - 0.5
    assert orc.Pi(h, A, xi) > 0
    # at the pole the averaged normal is -z by symmetry: repulsion pushes up
    assert fp[south, 2] > 0 and abs(fp[south, 0]) < 1e-14 and abs(fp[south, 1]) < 1e-14
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    At = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    chi_s = At[(tri == south).any(1)].sum()
    assert math.isclose(fp[south, 2], chi_s / 3.0 * orc.Pi(h, A, xi), rel_tol=1e-12)
    # at the top pole (normal +z) the slowly decaying attractive tail Pi < 0
    # gives -(chi/3) Pi n, i.e. a small outward push along +z
    top = int(np.argmax(xyz[:, 2]))
    ht = xyz[top, 2] - 0.5
    chi_t = At[(tri == top).any(1)].sum()
    assert orc.Pi(ht, A, xi) < 0
    assert math.isclose(fp[top, 2], -chi_t / 3.0 * orc.Pi(ht, A, xi), rel_tol=1e-12)


def test_near_wall_guard_counts_clamped_nodes(orc):
    xyz, tri = I.icosphere(2, 5.0, (10.0, 10.0, 0.5 + 5.0 + 0.2))
    A = orc.wetting_A(0.01, math.radians(90), 2.0)
    p = params(orc, sigma=0.01, wetting=1, A=A, xi=2.0, h_min_frac=0.5)
    _, _, fp, clamped = orc.membrane_forces(p, xyz, tri)
    h = xyz[:, 2] - 0.5
    assert clamped == int((h < 1.0).sum()) and clamped > 0
    assert np.all(np.isfinite(fp))


# ----------------------------------------------- elastic membrane (Skalak)
def fem_triangle_invariants(X0, X):
    """The invariants a, b of eq. strain_inv for one linear triangle, from the
    shape functions of Sec. II B as in fem_triangle_energy, and the
    reference area A0."""
    def frame(P):
        e1 = P[1] - P[0]
        n = np.cross(e1, P[2] - P[0])
        e1 = e1 / np.linalg.norm(e1)
        e2 = np.cross(n / np.linalg.norm(n), e1)
        return np.array([[(p - P[0]) @ e1, (p - P[0]) @ e2] for p in P])
    x0, x = frame(X0), frame(X)
    coef = np.linalg.inv(np.column_stack([x0, np.ones(3)]))
    D = np.eye(2) + (x - x0).T @ coef[:2, :].T
    Mdd = D @ D.T
    a = 0.5 * math.log(0.5 * np.trace(Mdd) ** 2 - 0.5 * np.trace(Mdd @ Mdd))
    b = 0.5 * np.trace(Mdd) - 1.0
    A0 = 0.5 * abs(np.linalg.det(np.column_stack([x0[1] - x0[0], x0[2] - x0[0]])))
    return a, b, A0


def skalak_energy(X0, X, ks, ka):
    """Skalak energy of a mesh triangle by triangle: A0 w with
    w = ks/12 (I1^2 + 2 I1 - 2 I2) + ka/12 I2^2, I1 = 2b, I2 = e^(2a) - 1."""
    a, b, A0 = fem_triangle_invariants(X0, X)
    I1, I2 = 2.0 * b, math.exp(2.0 * a) - 1.0
    return A0 * (ks / 12.0 * (I1 * I1 + 2.0 * I1 - 2.0 * I2) + ka / 12.0 * I2 * I2)


def test_skalak_invariants_match_principal_stretches():
    # a pure in-plane stretch by (l1, l2) of a right triangle: I1 = l1^2 +
    # l2^2 - 2 and I2 = l1^2 l2^2 - 1 (the Skalak invariants)
    X0 = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    l1, l2 = 1.3, 0.8
    X = X0 * np.array([l1, l2, 1.0])
    a, b, A0 = fem_triangle_invariants(X0, X)
    assert math.isclose(2 * b, l1 ** 2 + l2 ** 2 - 2, rel_tol=1e-12)
    assert math.isclose(math.exp(2 * a) - 1, l1 ** 2 * l2 ** 2 - 1, rel_tol=1e-12)
    assert math.isclose(A0, 0.5, rel_tol=1e-15)


def test_skalak_force_is_minus_energy_gradient(orc):
    xyz0, tri = I.icosphere(1, 3.0, (8.0, 8.0, 8.0))
    xyz = I.jitter_nodes(xyz0, 4, 0.25) * 1.05
    ks, ka = 0.04, 0.3
    p = params(orc, sigma=0.0, shear_modulus=ks, area_modulus=ka)
    phi = orc.membrane_elastic(p, xyz0, xyz, tri)
    h = 1e-6

    def energy(q):
        return sum(skalak_energy(xyz0[t], q[t], ks, ka) for t in tri)
    for j, a in ((0, 2), (7, 0), (23, 1), (41, 2)):
        xp, xm = xyz.copy(), xyz.copy()
        xp[j, a] += h
        xm[j, a] -= h
        assert abs(-(energy(xp) - energy(xm)) / (2 * h) - phi[j, a]) < 1e-7 * max(1.0, abs(phi[j, a]))


def test_skalak_force_vanishes_at_rest_and_under_rigid_motion(orc):
    xyz0, tri = jittered_sphere(level=2, seed=5)
    p = params(orc, sigma=0.0, shear_modulus=0.05, area_modulus=0.2)
    assert np.abs(orc.membrane_elastic(p, xyz0, xyz0, tri)).max() < 1e-13
    c, s = math.cos(0.7), math.sin(0.7)
    Rz = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    moved = xyz0 @ Rz.T + np.array([1.5, -2.0, 0.25])
    assert np.abs(orc.membrane_elastic(p, xyz0, moved, tri)).max() < 1e-12
    # a deformed state: no net force nor torque
    xyz = I.jitter_nodes(xyz0, 9, 0.3)
    phi = orc.membrane_elastic(p, xyz0, xyz, tri)
    assert np.abs(phi).max() > 1e-3
    assert np.allclose(phi.sum(0), 0.0, atol=1e-13)
    assert np.allclose(np.cross(xyz, phi).sum(0), 0.0, atol=1e-11)
    # zero moduli: no elastic force
    assert not orc.membrane_elastic(params(orc), xyz0, xyz, tri).any()
