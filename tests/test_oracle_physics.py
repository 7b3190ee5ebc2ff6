"""Physics pins of the oracle's full time step: Laplace pressure of a free
droplet (App. C: Delta p = 2 sigma / R_c without Pi), the ordering of the
equilibrium contact angle with theta_eq (Sec. II C: A sets the angle), mass
conservation with a membrane, the tau field for lambda != 1, the stored
statics trajectories' approach to the App. B equilibrium angle, and a
membrane carried by a uniform stream."""
import math
import os

import numpy as np
import pytest

from paper_2503_20605_gb300 import inputs as I


@pytest.mark.slow
def test_laplace_pressure_free_droplet(orc):
    n, R, sigma = 32, 8.0, 0.01
    xyz, tri = I.icosphere(3, R, (16.0, 16.0, 16.0))
    s = orc.Sim(orc.make_params(n, n, n, walls=0, tau_out=1.0, sigma=sigma))
    s.set_membrane(xyz, tri)
    s.step(1000)
    rho, u = s.macros()
    o = s.observe()
    Z, Y, X = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((X - o["cx"]) ** 2 + (Y - o["cy"]) ** 2 + (Z - o["cz"]) ** 2).ravel()
    dp = (rho[r < R - 3].mean() - rho[r > R + 3].mean()) / 3.0    # p = cs^2 rho
    RV = (3 * o["volume"] / (4 * math.pi)) ** (1 / 3)
    assert abs(dp / (2 * sigma / RV) - 1) < 0.03
    assert np.abs(u).max() < 1e-4        # spurious currents only


@pytest.mark.slow
def test_equilibrium_angle_follows_theta_eq(orc):
    """Droplets released at h = xi spread from the sphere (180 deg) towards
    their imposed angle: the measured angles keep the order of theta_eq."""
    got = []
    for th in (60.0, 120.0):
        sp = I.DropletSpec(24, 24, 18, 6.0, 3, 0.01, th, 1.5, tau=1.0)
        xyz, tri = sp.mesh()
        A = orc.wetting_A(sp.sigma, math.radians(th), sp.xi)
        s = orc.Sim(orc.make_params(24, 24, 18, tau_out=1.0, sigma=sp.sigma, wetting=1, A=A, xi=sp.xi,
                                    volume_correction=1))
        s.set_membrane(xyz, tri)
        s.step(1500)
        o = s.observe()
        assert s.clamped() == 0
        got.append(o["theta_RV"])
    assert got[0] < got[1] < 179.0
    assert got[1] - got[0] > 15.0


def test_mass_conserved_with_membrane(orc):
    sp = I.workload_parity_32()
    xyz, tri = sp.mesh()
    A = orc.wetting_A(sp.sigma, math.radians(sp.theta_deg), sp.xi)
    s = orc.Sim(orc.make_params(32, 32, 32, tau_out=1.0, sigma=sp.sigma, wetting=1, A=A, xi=sp.xi))
    s.set_membrane(xyz, tri)
    m0 = math.fsum(s.populations())
    s.step(20)
    assert abs(math.fsum(s.populations()) - m0) < 1e-13 * m0


def test_viscosity_ratio_sets_tau_inside(orc):
    sp = I.DropletSpec(24, 24, 24, 6.0, 3, 0.01, 90.0, 2.0, tau=0.8, lam=10.0)
    xyz, tri = sp.mesh()
    s = orc.Sim(orc.make_params(24, 24, 24, tau_out=sp.tau, tau_in=sp.tau_in, sigma=sp.sigma))
    s.set_membrane(xyz, tri)
    s.step(1)
    tau = s.tau()
    n_in = int((tau == sp.tau_in).sum())
    assert math.isclose(sp.tau_in, 0.5 + 10 * 0.3)
    assert set(np.unique(tau)) == {sp.tau, sp.tau_in}
    # the inside cells fill the droplet volume up to the surface discretisation
    assert abs(n_in / orc.mesh_volume(xyz, tri) - 1) < 0.1


def test_stored_statics_trajectory_reaches_theory_angle():
    """The oracle's half-scale statics trajectories (the stored file the
    reduced-precision GPU runs are held to; 64^3, R = 12, xi = 2, five
    theta_eq, 20 000 steps) settle at the angle of the App. B equilibrium at
    xi / R_V (R_V the radius of the sphere of the droplet's volume).  Each
    angle never rises (it stays at 180 degrees until the drop first touches
    the wall), and its changes per 1000 steps shrink steadily to below 0.1
    degree by the end; Aitken's delta-squared extrapolation of the last three
    samples then lands within 2 degrees of the theory's angle, and the limits
    keep the order of theta_eq.  Measured gaps, limit minus theory: -1.6,
    -0.8, -0.3, 0.0 and +0.1 degrees for theta_eq = 30 ... 150: the discrete
    droplet (L4 mesh, R = 12, xi / R0 = 0.17) settles a little flatter than
    the continuum theory at acute angles, where App. C also finds the
    weakest agreement between imposed and measured angles."""
    import oracle.shape as S
    d = np.loadtxt(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "statics64_oracle.txt"))
    limits = []
    for th in (30.0, 60.0, 90.0, 120.0, 150.0):
        r = d[d[:, 0] == th]
        assert r[-1, 1] == 20000
        a = r[:, 7]                                  # theta_RV, degrees
        assert np.all(np.diff(a) <= 0) and np.all(np.diff(a[-6:]) < 0), (th, a)
        d5 = np.diff(a[-6:])
        assert np.all(np.abs(d5[1:]) < np.abs(d5[:-1])), (th, d5)    # decelerating
        assert abs(d5[-1]) < 0.1, (th, d5)
        d1 = d5[-2:]
        lim = a[-1] - d1[1] ** 2 / (d1[1] - d1[0])
        rv = (3.0 * r[-1, 2] / (4.0 * math.pi)) ** (1.0 / 3.0)
        u, g, _, _ = S.solve(math.radians(th), 2.0 / rv, n_grid=801)
        theo = math.degrees(S.angle_from_height(g))
        assert abs(lim - theo) <= 2.0, (th, lim, theo)
        assert lim < a[-1]
        limits.append(lim)
    assert np.all(np.diff(limits) > 0), limits


def test_membrane_carried_by_uniform_stream(orc):
    """Without surface tension or wetting nothing forces the fluid, a
    uniform stream U stays uniform, the interpolated node velocity is U
    (eq. vel_interpolation; the kernel sums to one) and each forward-Euler
    update of the node positions (Sec. II A, dt = 1) moves every node by
    exactly U."""
    n, U, steps = 16, np.array([0.03, -0.02, 0.01]), 50
    xyz, tri = I.icosphere(2, 4.0, (8.0, 8.0, 8.0))
    s = orc.Sim(orc.make_params(n, n, n, walls=0, tau_out=0.9, sigma=0.0))
    s.set_populations(np.repeat(orc.feq(1.0, U)[:, None], n ** 3, axis=1).ravel())
    s.set_membrane(xyz, tri)
    s.step(steps)
    assert np.allclose(s.nodes(), xyz + steps * U, rtol=0, atol=1e-11)
