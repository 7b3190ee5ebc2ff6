"""The Python binding's view of the C ABI matches include/iblb.h, checked by
the C compiler itself (no GPU, no CUDA): a small C program includes the
header and prints the size of each descriptor struct and the offset of each
field, and every integer constant the header defines; the ctypes structures
and the constants of paper_2503_20605_gb300/iblb.py must agree with them.
A field added to a header struct without its binding (or in another order)
would otherwise shift every later field silently.  The oracle's binding of
oracle/oracle.h is checked the same way."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2503_20605_gb300 import iblb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "iblb.h")

# C struct name -> (ctypes structure, C field name of each ctypes field)
STRUCTS = {
    "iblb_lattice_desc": (iblb.LatticeDesc, {"lambda_": "lambda"}),
    "iblb_physics_desc": (iblb.PhysicsDesc, {}),
    "iblb_obs": (iblb.Obs, {}),
}


def header_constants():
    src = open(HEADER).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (IBLB_\w+)\s+(-?\d+)\b", src, re.M)}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "iblb.h"', "int main(void) {"]
    for cname, (cls, rename) in STRUCTS.items():
        lines.append(f'    printf("size {cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            cf = rename.get(f, f)
            lines.append(f'    printf("off {cname} {f} %zu\\n", offsetof({cname}, {cf}));')
    for name in header_constants():
        lines.append(f'    printf("const {name} %d\\n", (int)({name}));')
    lines += ["    return 0;", "}"]
    src, exe = d / "abi.c", d / "abi"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    size, off, const = {}, {}, {}
    for line in out.splitlines():
        kind, *rest = line.split()
        if kind == "size":
            size[rest[0]] = int(rest[1])
        elif kind == "off":
            off[(rest[0], rest[1])] = int(rest[2])
        else:
            const[rest[0]] = int(rest[1])
    return size, off, const


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_header(c_layout, cname):
    size, off, _ = c_layout
    cls, _ = STRUCTS[cname]
    assert C.sizeof(cls) == size[cname], cname
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == off[(cname, f)], (cname, f)


def test_struct_fields_are_all_bound():
    # every member the header declares in a descriptor struct has a ctypes
    # field: count the declarators between the braces of each typedef
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for cname, (cls, rename) in STRUCTS.items():
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + cname + r"\s*;", src).group(1)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # "double zmin, zmax" -> zmin, zmax; "double centroid[3]" -> centroid
            parts = decl.split(None, 1)[1]
            names += [re.sub(r"\[.*\]", "", p).strip() for p in parts.split(",")]
        bound = [rename.get(f, f) for f, _ in cls._fields_]
        assert bound == names, (cname, bound, names)


def test_constants_match_header(c_layout):
    _, _, const = c_layout
    for name, v in const.items():
        if name == "IBLB_H":
            continue
        assert hasattr(iblb, name), name
        assert getattr(iblb, name) == v, (name, getattr(iblb, name), v)
    assert set(iblb.CODE_NAMES) == {v for k, v in const.items() if k == "IBLB_OK" or k.startswith("IBLB_E_")}


def test_oracle_binding_matches_its_header(tmp_path):
    """The same check for the oracle's ctypes view of oracle/oracle.h: the
    parameter struct's layout and the order of the observables array."""
    import oracle.oracle as O
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "oracle.h"', "int main(void) {",
             '    printf("size %zu\\n", sizeof(orc_params));']
    for f, _ in O.Params._fields_:
        lines.append(f'    printf("off {f} %zu\\n", offsetof(orc_params, {f}));')
    for k, name in enumerate(O.OBS_NAMES):
        lines.append(f'    printf("obs {name} %d\\n", (int)ORC_OBS_{name.upper()});')
    lines.append('    printf("nobs %d\\n", (int)ORC_OBS_N);')
    lines += ["    return 0;", "}"]
    src, exe = tmp_path / "orc_abi.c", tmp_path / "orc_abi"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "oracle"), "-o", str(exe),
                    str(src)], check=True, capture_output=True)
    out = [ln.split() for ln in subprocess.run([str(exe)], check=True, capture_output=True,
                                               text=True).stdout.splitlines()]
    got = {(r[0], r[1]) if len(r) == 3 else (r[0],): int(r[-1]) for r in out}
    assert C.sizeof(O.Params) == got[("size",)]
    for f, _ in O.Params._fields_:
        assert getattr(O.Params, f).offset == got[("off", f)], f
    for k, name in enumerate(O.OBS_NAMES):
        assert got[("obs", name)] == k, name
    assert got[("nobs",)] == len(O.OBS_NAMES)
