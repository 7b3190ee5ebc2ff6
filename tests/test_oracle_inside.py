"""Pins of the oracle's in/out classification used for tau(x) (Sec. II A:
tau_in inside the closed interface, tau_out outside, identified by ray
tracing).  The reference is the generalized winding number (sum of signed
solid angles / 4 pi), which is 1 inside and 0 outside a closed outward mesh
independently of any ray; and watertightness on meshes whose vertices and
edges sit exactly on lattice columns."""
import numpy as np
import pytest

from paper_2503_20605_gb300 import inputs as I


def winding_number(xyz, tri, P):
    """Van Oosterom-Strackee solid angles summed over faces, / 4 pi."""
    out = np.zeros(len(P))
    for k0 in range(0, len(P), 2048):
        p = P[k0:k0 + 2048, None, :]
        a, b, c = xyz[tri[:, 0]] - p, xyz[tri[:, 1]] - p, xyz[tri[:, 2]] - p
        la, lb, lc = (np.linalg.norm(v, axis=2) for v in (a, b, c))
        num = np.einsum("pfk,pfk->pf", a, np.cross(b, c))
        den = la * lb * lc + np.einsum("pfk,pfk->pf", a, b) * lc + \
            np.einsum("pfk,pfk->pf", a, c) * lb + np.einsum("pfk,pfk->pf", b, c) * la
        out[k0:k0 + 2048] = (2.0 * np.arctan2(num, den)).sum(1) / (4 * np.pi)
    return out


def cell_points(nx, ny, nz, walls):
    z0 = 1 if walls else 0
    nzf = nz - 2 if walls else nz
    Z, Y, X = np.meshgrid(np.arange(z0, z0 + nzf), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(float)


def surface_distance_ok(xyz, tri, P, tol):
    """points farther than tol from every vertex and face plane patch
    (cheap conservative filter: distance to vertices and to face centroids)."""
    cen = xyz[tri].mean(1)
    dv = np.min(np.linalg.norm(P[:, None, :] - xyz[None], axis=2), axis=1)
    dc = np.min(np.linalg.norm(P[:, None, :] - cen[None], axis=2), axis=1)
    return (dv > tol) & (dc > tol)


@pytest.mark.parametrize("center,level", [((10.3, 9.7, 9.9), 2), ((10.0, 10.0, 10.0), 2),
                                          ((9.5, 10.5, 10.0), 3)])
def test_inside_matches_winding_number_sphere(orc, center, level):
    nx = ny = nz = 20
    xyz, tri = I.icosphere(level, 6.0, center)
    p = orc.make_params(nx, ny, nz, walls=1)
    ins = orc.inside(p, xyz, tri)
    P = cell_points(nx, ny, nz, 1)
    w = winding_number(xyz, tri, P)
    edge = np.linalg.norm(xyz[tri[:, 0]] - xyz[tri[:, 1]], axis=1).max()
    ok = surface_distance_ok(xyz, tri, P, 0.5 * edge)
    assert ok.sum() > 0.8 * len(P)
    assert np.all(np.abs(w[ok] - np.round(w[ok])) < 1e-9)
    assert np.array_equal(ins[ok].astype(bool), (w[ok] > 0.5))
    # even crossing count in every column: the top fluid layer is outside
    assert not ins.reshape(nz - 2, ny, nx)[-1].any()


def cube(lo, hi):
    v = np.array([[x, y, z] for z in (lo, hi) for y in (lo, hi) for x in (lo, hi)], float)
    # outward CCW faces of the cube with corner index x + 2y + 4z
    f = [(0, 2, 1), (1, 2, 3), (4, 5, 6), (5, 7, 6), (0, 1, 4), (1, 5, 4),
         (2, 6, 3), (3, 6, 7), (0, 4, 2), (2, 4, 6), (1, 3, 5), (3, 7, 5)]
    return v, np.array(f, np.int32)


def octahedron(c, r):
    c = np.asarray(c, float)
    v = np.array([c + [r, 0, 0], c - [r, 0, 0], c + [0, r, 0], c - [0, r, 0], c + [0, 0, r], c - [0, 0, r]])
    f = [(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4), (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)]
    return v, np.array(f, np.int32)


@pytest.mark.parametrize("mesh", ["cube", "octahedron"])
def test_inside_watertight_on_lattice_aligned_meshes(orc, mesh):
    """Vertices and edges exactly on columns, vertical faces with zero
    projected area: every column must still see an even number of crossings,
    cells strictly inside / outside must be classified as the closed-form
    solid says, and cells on the surface are assigned by the half-open rule."""
    nx = ny = nz = 14
    P = cell_points(nx, ny, nz, 1)
    if mesh == "cube":
        xyz, tri = cube(3.0, 9.0)
        dist = np.max(np.abs(P - 6.0), axis=1) - 3.0         # < 0 inside, 0 on the surface
    else:
        xyz, tri = octahedron((7.0, 7.0, 6.0), 4.0)
        dist = np.abs(P - [7.0, 7.0, 6.0]).sum(1) - 4.0
    assert orc.mesh_volume(xyz, tri) > 0
    p = orc.make_params(nx, ny, nz, walls=1)
    ins = orc.inside(p, xyz, tri)
    assert np.all(ins[dist < 0] == 1) and np.all(ins[dist > 0] == 0)
    col = ins.reshape(nz - 2, -1)
    assert not col[-1].any() and not col[0].any()
    # each column holds one contiguous run of inside cells at most
    for c in col.T:
        d = np.diff(np.concatenate([[0], c, [0]]).astype(int))
        assert (d == 1).sum() <= 1
    if mesh == "cube":
        # the half-open rule keeps exactly one of the two bounding planes per axis
        assert ins.sum() == 6 * 6 * 6


def test_inside_periodic_image(orc):
    """A mesh that straddles the x seam is classified through its periodic
    image (columns are wrapped)."""
    nx = ny = nz = 16
    xyz, tri = I.icosphere(2, 4.0, (15.2, 8.3, 7.9))
    p = orc.make_params(nx, ny, nz, walls=1)
    ins = orc.inside(p, xyz, tri).reshape(nz - 2, ny, nx)
    xyz2 = xyz.copy()
    xyz2[:, 0] -= 8.0
    ins2 = orc.inside(p, xyz2, tri).reshape(nz - 2, ny, nx)
    assert ins.sum() == ins2.sum() > 0
    assert np.array_equal(np.roll(ins2, 8, axis=2), ins)
