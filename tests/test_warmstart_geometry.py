"""The warm start's mesh geometry: the FP64 oracle (oracle/warmstart.py)
pinned against closed forms -- a sphere has g = 1, an exact spherical cap
has the App. B volume constraint (integral of g^3 sin(phi) = 2, eq.
volconstr2) and the hemisphere's closed-form heights -- and the library's
host functions iblb_mesh_profile / iblb_deform_mesh against the oracle.
No GPU is needed: both library calls are host code."""
import numpy as np
import pytest

import oracle.warmstart as W
from paper_2503_20605_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    from paper_2503_20605_gb300 import build
    build.build()
    from paper_2503_20605_gb300 import iblb
    return iblb


def test_sphere_profile_is_one():
    xyz, _ = I.icosphere(4, 7.5, (0.0, 0.0, 0.0))
    np.testing.assert_allclose(W.profile(xyz, 7.5), 1.0, atol=1e-12)


@pytest.mark.parametrize("theta_deg", [20, 45, 90, 135, 160])
def test_cap_profile_volume_constraint(theta_deg):
    n = 4000
    g = W.cap_profile(np.radians(theta_deg), n)
    phi = (np.arange(n) + 0.5) * np.pi / n
    assert abs(np.sum(g ** 3 * np.sin(phi)) * np.pi / n - 2.0) < 2e-3


def test_hemisphere_closed_form():
    rho = 2.0 ** (1.0 / 3.0)           # hemisphere of volume 4 pi / 3
    g = W.cap_profile(np.pi / 2, 4000)
    # surface centroid at rho / 3 above the base: straight up rho - rho/3, straight down rho/3
    assert abs(g[0] - 2 * rho / 3) < 1e-5 and abs(g[-1] - rho / 3) < 1e-5


def test_deform_identity_and_invariants():
    xyz, tri = I.icosphere(4, 10.0, (0.0, 0.0, 0.0))
    out = W.deform(np.ones(64), 10.0, xyz, tri, 5.0, 6.0, 2.5)
    # the sphere maps onto itself up to the area quadrature (4096 intervals)
    np.testing.assert_allclose(out, xyz + np.array([5.0, 6.0, 12.5]), atol=1e-5)
    g = 1.0 + 0.25 * np.cos(2 * (np.arange(64) + 0.5) * np.pi / 64)
    out = W.deform(g, 10.0, xyz, tri, 5.0, 6.0, 2.5)
    assert abs(W.mesh_volume(out, tri) / W.mesh_volume(xyz, tri) - 1.0) < 1e-13
    assert abs(out[:, 2].min() - 2.5) < 1e-13
    # the profile of the deformed mesh follows g up to the volume rescaling
    # and the binning (the shape is symmetric, so the node centroid stays put)
    gp = W.profile(out, 10.0)
    n = 4000
    phi = (np.arange(n) + 0.5) * np.pi / n
    gf = 1.0 + 0.25 * np.cos(2 * phi)
    s = np.cbrt(2.0 / (np.sum(gf ** 3 * np.sin(phi)) * np.pi / n))   # eq. volconstr2 rescaling
    assert np.max(np.abs(gp - s * g)) < 0.01


def test_library_matches_oracle(lib):
    rng = np.random.default_rng(3)
    xyz, tri = I.icosphere(3, 9.0, (20.0, 21.0, 12.0))
    g = W.cap_profile(np.radians(70.0), 64) * (1 + 0.01 * rng.standard_normal(64))
    out_l = lib.iblb_deform_mesh(g, 9.0, xyz, tri, 30.0, 31.0, 2.5)
    out_o = W.deform(g, 9.0, xyz, tri, 30.0, 31.0, 2.5)
    np.testing.assert_allclose(out_l, out_o, rtol=0, atol=1e-11)
    np.testing.assert_allclose(lib.iblb_mesh_profile(out_l, 9.0), W.profile(out_l, 9.0), rtol=0, atol=1e-12)
    # a coarse mesh leaves bins empty: interpolated alike
    small, _ = I.icosphere(1, 3.0, (0.0, 0.0, 0.0))
    np.testing.assert_allclose(lib.iblb_mesh_profile(small, 3.0, 64), W.profile(small, 3.0, 64), atol=1e-12)


def test_library_rejects_bad_input(lib):
    xyz, tri = I.icosphere(2, 5.0, (0.0, 0.0, 0.0))
    with pytest.raises(lib.IblbError) as e:
        lib.iblb_deform_mesh(-np.ones(64), 5.0, xyz, tri, 0, 0, 0)
    assert e.value.code == lib.IBLB_E_ARG
    with pytest.raises(lib.IblbError) as e:
        lib.iblb_deform_mesh(np.ones(64), 5.0, xyz, np.where(tri == 3, 10 ** 6, tri), 0, 0, 0)
    assert e.value.code == lib.IBLB_E_MESH
    with pytest.raises(lib.IblbError) as e:
        lib.iblb_mesh_profile(np.zeros((4, 3)), 1.0)
    assert e.value.code == lib.IBLB_E_MESH


def _face_areas(q, tri):
    a, b, c = q[tri[:, 0]], q[tri[:, 1]], q[tri[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def test_equal_area_map_keeps_faces_even():
    """On a flat cap (theta = 30 deg) the area-preserving placement keeps the
    face areas far more even than moving each node radially."""
    xyz, tri = I.icosphere(4, 10.0, (0.0, 0.0, 0.0))
    g = W.cap_profile(np.radians(30.0), 64)
    ours = W.deform(g, 10.0, xyz, tri, 0.0, 0.0, 0.0)
    r = np.linalg.norm(xyz, axis=1)
    radial = (10.0 * W.profile_at(g, np.arccos(np.clip(xyz[:, 2] / r, -1, 1))) / r)[:, None] * xyz
    cv = lambda q: np.std(_face_areas(q, tri)) / np.mean(_face_areas(q, tri))
    assert cv(ours) < 0.5 * cv(radial), (cv(ours), cv(radial))


@pytest.mark.parametrize("theta_deg", [20, 45, 90, 135, 160])
def test_package_cap_profile_equals_oracle(theta_deg):
    # the spherical-cap start of the package (paper_2503_20605_gb300.warmstart)
    # against the oracle's exact cap, which the volume constraint pins above
    from paper_2503_20605_gb300 import warmstart as PW
    np.testing.assert_allclose(PW.cap_profile(theta_deg), W.cap_profile(np.radians(theta_deg), 64),
                               rtol=1e-12, atol=1e-12)
