"""Pins of the oracle's observables: angle from height (App. C, eqs. ell,
voldrop, angleh), contact radius protocols (i) and (ii) (Sec. III B) and
the volume correction of the time step."""
import math

import numpy as np
import pytest

from paper_2503_20605_gb300 import inputs as I


@pytest.mark.parametrize("theta_deg", [10, 30, 45, 60, 90, 120, 150, 170])
def test_angle_from_height_inverts_spherical_cap(orc, theta_deg):
    """A spherical cap of radius Rc meeting the wall at theta has height
    H = Rc (1 - cos theta) and volume pi H^2 (3 Rc - H) / 3; with R0 the
    radius of the sphere of equal volume and l = H/2, eq. angleh returns theta."""
    th = math.radians(theta_deg)
    Rc = 3.7
    H = Rc * (1 - math.cos(th))
    V = math.pi * H * H * (3 * Rc - H) / 3
    R0 = (3 * V / (4 * math.pi)) ** (1 / 3)
    assert math.isclose(orc.theta_from_height(H / 2, R0), th, rel_tol=1e-12)
    # eq. ell: l = Rc sin^2(theta/2); eq. contactr: r_c = Rc sin(theta)
    assert math.isclose(H / 2, Rc * math.sin(th / 2) ** 2, rel_tol=1e-12)
    rc = Rc * math.sin(th)
    # eq. voldrop: 8 R0^3 / r_c^3 = tan(theta/2) (3 + tan^2(theta/2))
    t = math.tan(th / 2)
    assert math.isclose(8 * R0 ** 3 / rc ** 3, t * (3 + t * t), rel_tol=1e-12)


def test_sphere_observables(orc):
    R = 9.0
    xyz, tri = I.icosphere(5, R, (20.0, 21.0, 12.0))
    V = orc.mesh_volume(xyz, tri)
    R0 = (3 * V / (4 * math.pi)) ** (1 / 3)
    o = orc.mesh_observe(xyz, tri, R0, zcut_frac=0.5, eps_flat=0.1)
    assert math.isclose(o["volume"], 4 / 3 * math.pi * R ** 3, rel_tol=2e-3)
    assert math.isclose(o["area"], 4 * math.pi * R ** 2, rel_tol=2e-3)
    assert np.allclose([o["cx"], o["cy"], o["cz"]], [20.0, 21.0, 12.0], atol=1e-9)
    assert math.isclose(o["zmax"] - o["zmin"], 2 * R, rel_tol=1e-12)
    assert o["theta_R0"] == 180.0
    # protocol (i): plane at z_wall + 0.5 R0 cuts the sphere in a circle
    zp = 0.5 + 0.5 * R0
    d = 12.0 - zp
    assert o["n_cut"] > 50
    assert math.isclose(o["rc_cut"], math.sqrt(R * R - d * d), rel_tol=5e-3)


def test_flat_bottom_protocol_ii(orc):
    """Flatten the lower part of a sphere onto z = z0: the flat triangles in
    the lower half cover (up to the ragged rim) the disk of radius
    sqrt(R^2 - (zc - z0)^2), so r_eps approaches that radius."""
    R, zc = 10.0, 14.0
    xyz, tri = I.icosphere(5, R, (30.0, 30.0, zc))
    z0 = zc - 0.6 * R
    xyz[:, 2] = np.maximum(xyz[:, 2], z0)
    V = orc.mesh_volume(xyz, tri)
    R0 = (3 * V / (4 * math.pi)) ** (1 / 3)
    o = orc.mesh_observe(xyz, tri, R0, zcut_frac=0.05, eps_flat=0.01)
    r_disk = math.sqrt(R * R - (zc - z0) ** 2)
    assert abs(o["rc_flat"] / r_disk - 1) < 0.03
    assert math.isclose(o["chi_flat"], math.pi * o["rc_flat"] ** 2, rel_tol=1e-12)


def test_volume_correction_holds_volume(orc):
    sp = I.workload_parity_32()
    xyz, tri = sp.mesh()
    A = orc.wetting_A(sp.sigma, math.radians(60.0), sp.xi)
    p = orc.make_params(32, 32, 32, tau_out=1.0, sigma=sp.sigma, wetting=1, A=A, xi=sp.xi,
                        volume_correction=1)
    s = orc.Sim(p)
    s.set_membrane(xyz, tri)
    V0 = orc.mesh_volume(xyz, tri)
    s.step(20)
    assert math.isclose(s.observe()["volume"], V0, rel_tol=1e-13)
    p0 = orc.make_params(32, 32, 32, tau_out=1.0, sigma=sp.sigma, wetting=1, A=A, xi=sp.xi)
    s0 = orc.Sim(p0)
    s0.set_membrane(xyz, tri)
    s0.step(20)
    assert not np.allclose(s0.nodes(), s.nodes(), atol=1e-12)


def _vc_pair(orc, shift):
    """One step from the same state, with and without the volume correction.
    The state is a droplet that has run 20 steps (so V != V0), placed
    `shift` cells along x and y in the periodic box."""
    sp = I.workload_parity_32()
    xyz, tri = sp.mesh()
    A = orc.wetting_A(sp.sigma, math.radians(60.0), sp.xi)
    kw = dict(tau_out=1.0, sigma=sp.sigma, wetting=1, A=A, xi=sp.xi)
    s = orc.Sim(orc.make_params(32, 32, 32, **kw))
    s.set_membrane(xyz, tri)
    s.step(20)
    f = s.populations().reshape(19, 30, 32, 32)      # [i][z][y][x], fluid layers only
    f = np.roll(f, (shift, shift), axis=(2, 3)).ravel()
    q = s.nodes() + [shift, shift, 0.0]
    out = []
    for vc in (0, 1):
        t = orc.Sim(orc.make_params(32, 32, 32, volume_correction=vc, **kw))
        t.set_membrane(xyz + [shift, shift, 0.0], tri)   # V0: the volume of the mesh as set
        t.set_populations(f)
        t.set_nodes(q)
        t.step(1)
        out.append(t.nodes())
    return out, orc.mesh_volume(xyz, tri), tri


def test_volume_correction_keeps_node_centroid(orc):
    """The correction rescales the mesh about its node centroid (a uniform
    dilation about c leaves c in place): one corrected step and one
    uncorrected step from the same state end with the same node centroid,
    to round-off, while the corrected mesh has the initial volume and the
    uncorrected one does not.  A dilation about another point (the origin,
    say) moves the centroid by (k - 1) times its distance from that point."""
    (q_off, q_on), V0, tri = _vc_pair(orc, 0)
    assert abs(orc.mesh_volume(q_off, tri) / V0 - 1.0) > 1e-7
    assert math.isclose(orc.mesh_volume(q_on, tri), V0, rel_tol=1e-13)
    assert np.abs(q_on.mean(axis=0) - q_off.mean(axis=0)).max() < 1e-12
    # the correction is a dilation: every node moves along its ray from c
    c = q_off.mean(axis=0)
    d_off, d_on = q_off - c, q_on - c
    k = (d_on * d_off).sum() / (d_off * d_off).sum()
    assert np.abs(d_on - k * d_off).max() < 1e-12
    assert abs(k ** 3 - V0 / orc.mesh_volume(q_off, tri)) < 1e-12


def test_volume_correction_commutes_with_translation(orc):
    """The step is translation invariant in the periodic directions, and so
    is a correction about the node centroid: the droplet moved by whole
    cells along x and y ends moved by the same amount, with the same shape,
    to round-off."""
    (_, q0), _, _ = _vc_pair(orc, 0)
    (_, q7), _, _ = _vc_pair(orc, 7)
    assert np.abs(q7 - [7.0, 7.0, 0.0] - q0).max() < 1e-11
