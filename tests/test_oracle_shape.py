"""Pins of the axisymmetric equilibrium-shape solver (oracle/shape.py, App.
B) against what the paper fixes independently of the solver: the exact
spherical cap eq. gcap solves eq. YL without the wall term (to the order of
the finite differences); the measured angle at theta_eq = pi/4, xi/R0 = 0.1
is the 0.32 pi printed in the caption of Fig. 8 (tests/golden/paper_fig8.txt);
the film gap matches the planar solution of App. C; the measured angle moves
toward the imposed one as xi/R0 decreases.

The 0.28 pi printed for xi/R0 = 0.01 is not used as a pin: on a grid graded
about the contact line the solution converges to 0.2544 pi there (801
points 0.2528 pi, 1601 points 0.2540 pi, 3201 points 0.2543 pi: second-order
convergence; uniform grids approach it from below, 0.2534 pi with 6401
points), in line with the
paper's statement that the measured angle tends to theta_eq as xi/R0 -> 0;
0.28 pi is what the solution gives at xi/R0 = 0.05.  The test below checks
that approach instead, and App. C's own structure arbitrates between the two
values: at xi/R0 = 0.01 the solution must be the cap of eq. gcap away from
the wall and the plane of eq. gplanar near u = -1, with c = 2/k from its own
pressure jump and the angle it measures by eq. angleh.  It is, to a few
parts in a thousand with the measured 0.253 pi; with 0.28 pi both forms miss
it by about a tenth of R0.  A cap of volume 4 pi/3 whose pressure jump is the
solution's (k = 0.779) meets the wall at 0.252 pi; 0.28 pi would need k =
0.885."""
import os

import numpy as np
import pytest

import oracle.shape as S

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_fig8.txt")


def _cap_residual(n_grid, theta):
    u = np.linspace(-1.0, 1.0, n_grid)
    g, c = S.cap_g(u, theta)
    x = np.concatenate([g, [0.0, 2.0 / c]])
    return np.max(np.abs(S.residual(x, u, 0.1, theta, wall=False)[:n_grid]))


@pytest.mark.parametrize("theta", [np.pi / 4, np.pi / 2, 3 * np.pi / 4])
def test_cap_solves_young_laplace_without_wall(theta):
    r1, r2 = _cap_residual(401, theta), _cap_residual(801, theta)
    assert r1 < 1e-3 and r2 < r1 / 3.5            # second-order convergence


@pytest.fixture(scope="module")
def sol_01():
    return S.solve(np.pi / 4, 0.1, n_grid=401)


def test_measured_angle_fig8(sol_01):
    rows = np.loadtxt(GOLD)
    want = rows[(rows[:, 0] == 0.25) & (rows[:, 1] == 0.1)][0, 2]
    u, g, delta, k = sol_01
    assert abs(S.angle_from_height(g) / np.pi - want) < 0.005
    assert abs(np.trapezoid(g ** 3, u) - 2.0) < 1e-10 and abs(g[0] - g[-1]) < 1e-12


def test_film_gap_matches_planar_solution(sol_01):
    u, g, delta, k = sol_01
    assert abs(delta / S.film_thickness(0.1, k, np.pi / 4) - 1.0) < 1e-4


def test_angle_moves_toward_imposed_as_eps_shrinks(sol_01):
    th01 = S.angle_from_height(sol_01[1])
    th005 = S.angle_from_height(S.solve(np.pi / 4, 0.05, n_grid=1601)[1])
    assert np.pi / 4 < th005 < th01


def test_profile_about_centroid_of_offset_sphere():
    # a sphere of radius a centred a height s above the origin: r(u) = s u +
    # sqrt(a^2 - s^2 (1 - u^2)); its centroid is its centre, about which the
    # profile is the constant a
    a, s = 1.3, -0.55
    u = np.linspace(-1.0, 1.0, 4001)
    r = s * u + np.sqrt(a * a - s * s * (1.0 - u * u))
    assert abs(S.centroid_height(u, r) - s) < 1e-6
    phi = np.linspace(0.0, np.pi, 97)
    assert np.abs(S.profile_about_centroid(u, r, phi) - a).max() < 1e-6


def test_profile_about_centroid_of_hemisphere():
    # a unit hemisphere, flat face down at z = -1/2 (origin at mid-height):
    # centroid 3/8 above the flat face, so the top is 5/8 and the bottom
    # 3/8 away from it, and the rim at sqrt(1 + (3/8)^2)
    u = np.linspace(-1.0, 1.0, 20001)
    # ray from (0, 0) along (sqrt(1-u^2), u) hits the sphere x^2 + (z + 1/2)^2 = 1
    # (for z >= -1/2) or the plane z = -1/2
    b = 0.5 * u
    t_sph = -b + np.sqrt(b * b + 0.75)
    with np.errstate(divide="ignore"):
        t_pl = np.where(u < 0, -0.5 / np.where(u < 0, u, -1.0), np.inf)
    r = np.minimum(t_sph, t_pl)
    zc = S.centroid_height(u, r)
    assert abs(zc - (-0.5 + 0.375)) < 1e-4
    G = S.profile_about_centroid(u, r, np.array([0.0, np.pi]))
    assert abs(G[0] - 0.625) < 1e-4 and abs(G[1] - 0.375) < 1e-4


def test_graded_grid_agrees_and_angle_approaches_imposed():
    # where the uniform grid converges (xi/R0 = 0.05) the graded one agrees
    th05 = S.angle_from_height(S.solve_graded(np.pi / 4, 0.05, n_grid=801)[1])
    assert abs(th05 - S.angle_from_height(S.solve(np.pi / 4, 0.05, n_grid=1601)[1])) < 1e-3 * np.pi
    # at xi/R0 = 0.01 the measured angle is within a fifth of the xi/R0 = 0.1
    # bias of theta_eq (App. C: theta -> theta_eq as xi/R0 -> 0)
    th01 = S.angle_from_height(S.solve_graded(np.pi / 4, 0.01, n_grid=801)[1])
    th10 = S.angle_from_height(S.solve(np.pi / 4, 0.1, n_grid=401)[1])
    assert np.pi / 4 < th01 < th05 < th10
    assert th01 - np.pi / 4 < 0.2 * (th10 - np.pi / 4)



@pytest.fixture(scope="module")
def sol_001():
    return S.solve_graded(np.pi / 4, 0.01, n_grid=801)


def _gcap(u, c, th):
    C2 = np.cos(th / 2) ** 2
    return c * (-C2 * u + np.sqrt(1.0 - C2 * C2 * (1.0 - u * u)))


def _gplanar(u, c, th):
    return -c * np.sin(th / 2) ** 2 / u


def test_app_c_structure_at_eps_001(sol_001):
    """App. C at theta_eq = pi/4, xi/R0 = 0.01 (Fig. 9).  Away from the wall
    the solution of eq. YL is the spherical cap eq. gcap of radius c = 2/k
    (its Laplace pressure) meeting the wall at the angle measured by eq.
    angleh; near u = -1 it is the plane eq. gplanar, z = -c sin^2(theta/2);
    the film under it has the planar gap of App. C.  The cap radius is tied
    to the pressure jump k and the angle to the half-height, so the check
    involves the wall term (through k and the gap) and the curvature (through
    the cap) independently of the solver."""
    u, g, delta, k = sol_001
    c = 2.0 / k
    th = S.angle_from_height(g)
    cap, flat = u >= 0.0, u <= -0.95
    assert np.abs(g[cap] - _gcap(u[cap], c, th)).max() < 1e-2
    assert np.abs(g[flat] - _gplanar(u[flat], c, th)).max() < 5e-3
    # the cap radius from the half-height (eq. ell) against 2/k: O(eps)
    assert abs(g[-1] / np.sin(th / 2) ** 2 / c - 1.0) < 0.015
    assert abs(delta / S.film_thickness(0.01, k, np.pi / 4) - 1.0) < 1e-5
    # the printed 0.28 pi does not fit the same structure
    th_p = 0.28 * np.pi
    assert np.abs(g[cap] - _gcap(u[cap], c, th_p)).max() > 0.1
    assert np.abs(g[flat] - _gplanar(u[flat], c, th_p)).max() > 0.05
