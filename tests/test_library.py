"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every function include/iblb.h declares; the Python binding
covers each of them; argument validation that happens before any CUDA call
returns IBLB_E_ARG; host parameter helpers agree with the oracle."""
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
