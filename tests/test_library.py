"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every function include/iblb.h declares; the Python binding
covers each of them; argument validation that happens before any CUDA call
returns IBLB_E_ARG; host parameter helpers agree with the oracle; the
host-only mesh check accepts closed meshes with their exact volume and
refuses every kind of broken mesh with IBLB_E_MESH."""
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_20605_gb300 import build
    build.build()
    from paper_2503_20605_gb300 import iblb
    return iblb


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(iblb_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_api():
    names = declared_functions()
    for n in ("iblb_create", "iblb_step", "iblb_set_membrane", "iblb_get_populations", "iblb_get_nodes",
              "iblb_observe", "iblb_batch_create", "iblb_destroy", "iblb_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in sorted(declared_functions()):
        assert hasattr(so, n), n
    assert declared_functions() <= set(lib.exported_symbols())


def test_descriptor_validation_needs_no_gpu(lib):
    bad = [lib.lattice_desc(32, 32, 32, tau_out=0.5), lib.lattice_desc(4, 32, 32),
           lib.lattice_desc(32, 32, 32, lam=0.0), lib.lattice_desc(32, 32, 32, storage=7)]
    for d in bad:
        with pytest.raises(lib.IblbError) as e:
            lib.iblb_create(d, lib.physics_desc())
        assert e.value.code == lib.IBLB_E_ARG
    with pytest.raises(lib.IblbError) as e:
        lib.iblb_create(lib.lattice_desc(32, 32, 32), lib.physics_desc(sigma=0.01, theta_eq_deg=90.0, xi=-1.0))
    assert e.value.code == lib.IBLB_E_ARG
    with pytest.raises(lib.IblbError) as e:
        lib.iblb_create(lib.lattice_desc(32, 32, 32, walls=0), lib.physics_desc(theta_eq_deg=90.0))
    assert e.value.code == lib.IBLB_E_ARG
    mixed = [lib.lattice_desc(32, 32, 32, storage="f16"), lib.lattice_desc(32, 32, 32, storage="f32")]
    with pytest.raises(lib.IblbError):
        lib.iblb_batch_create(mixed, [lib.physics_desc(), lib.physics_desc()])


def test_wetting_A_matches_oracle(lib, orc):
    for th in (20.0, 45.0, 90.0, 150.0, 180.0):
        a = lib.iblb_wetting_A(0.013, th, 2.4, 6, 3)
        b = orc.wetting_A(0.013, math.radians(th), 2.4, 6, 3)
        assert math.isclose(a, b, rel_tol=1e-14, abs_tol=1e-18)
    with pytest.raises(lib.IblbError):
        lib.iblb_wetting_A(0.01, 90.0, 0.0)


def octahedron():
    """Vertices at +-1 on the axes, faces oriented outward: volume 4/3."""
    import numpy as np
    xyz = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)
    tri = []
    for a in (0, 1):
        for b in (2, 3):
            for c in (4, 5):
                t = [a, b, c]
                n = np.cross(xyz[b] - xyz[a], xyz[c] - xyz[a])
                tri.append(t if n @ (xyz[a] + xyz[b] + xyz[c]) > 0 else [a, c, b])
    return xyz, np.array(tri, np.int32)


def torus(n=12, m=8, R=3.0, r=1.0):
    """A closed, consistently oriented torus mesh (Euler characteristic 0)."""
    import numpy as np
    u, v = np.meshgrid(np.arange(n) * 2 * math.pi / n, np.arange(m) * 2 * math.pi / m, indexing="ij")
    xyz = np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], -1)
    idx = lambda i, j: (i % n) * m + (j % m)
    tri = []
    for i in range(n):
        for j in range(m):
            tri += [[idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)], [idx(i, j), idx(i + 1, j + 1), idx(i, j + 1)]]
    return xyz.reshape(-1, 3), np.array(tri, np.int32)


def test_check_mesh_accepts_closed_meshes(lib, orc):
    # the octahedron's volume is 4/3 exactly; an icosphere's equals the
    # oracle's divergence-theorem volume and lies below the sphere's
    xyz, tri = octahedron()
    assert math.isclose(lib.iblb_check_mesh(xyz, tri), 4.0 / 3.0, rel_tol=1e-15)
    from paper_2503_20605_gb300 import inputs as I
    xyz, tri = I.icosphere(3, 5.0, (10.0, 11.0, 12.0))
    v = lib.iblb_check_mesh(xyz, tri)
    assert math.isclose(v, orc.mesh_volume(xyz, tri), rel_tol=1e-13)
    assert 0.97 * 4 / 3 * math.pi * 125 < v < 4 / 3 * math.pi * 125


def test_check_mesh_refuses_what_set_membrane_refuses(lib):
    import numpy as np
    from paper_2503_20605_gb300 import inputs as I
    xyz, tri = I.icosphere(2, 5.0)
    one_flipped = tri.copy()
    one_flipped[7] = one_flipped[7, ::-1]
    t_xyz, t_tri = torus()
    o_xyz, o_tri = octahedron()
    two = (np.vstack([o_xyz, o_xyz + 5.0]), np.vstack([o_tri, o_tri + len(o_xyz)]))
    degenerate = tri.copy()
    degenerate[0, 1] = degenerate[0, 0]
    nan = xyz.copy()
    nan[3, 1] = np.nan
    bad = {
        "open": (xyz, tri[1:], "open mesh"),
        "inward": (xyz, tri[:, ::-1], "volume not positive"),
        "one face flipped": (xyz, one_flipped, "same direction"),
        "index out of range": (xyz, np.where(tri == 5, len(xyz), tri), "out of range"),
        "degenerate face": (xyz, degenerate, "degenerate"),
        "unused node": (np.vstack([xyz, [[0.0, 0.0, 9.0]]]), tri, "not used"),
        "torus": (t_xyz, t_tri, "Euler"),
        "two spheres": (two[0], two[1], "Euler"),
        "non-finite": (nan, tri, "non-finite"),
        "too small": (xyz[:3], np.array([[0, 1, 2]], np.int32), "at least 4"),
    }
    for name, (x, t, why) in bad.items():
        with pytest.raises(lib.IblbError) as e:
            lib.iblb_check_mesh(x, t)
        assert e.value.code == lib.IBLB_E_MESH, name
        assert why in str(e.value), (name, str(e.value))
    assert lib.lib().iblb_check_mesh(None, 4, None, 4, None) == lib.IBLB_E_ARG
