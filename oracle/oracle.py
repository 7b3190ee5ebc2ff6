"""ctypes binding of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  It never imports the CUDA package and
the CUDA package never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

OBS_NAMES = ["mass", "volume", "area", "cx", "cy", "cz", "zmin", "zmax", "theta_R0",
             "theta_RV", "rc_cut", "rc_flat", "n_cut", "chi_flat"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc, plain IEEE FP64)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        tmp = LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC", "-shared"]
        # OpenMP shares the independent cells of the stream-collide loop among
        # threads (same bits as one thread); plain build where it is missing
        if subprocess.run(base + ["-fopenmp", "-o", tmp, SRC, "-lm"], capture_output=True).returncode:
            subprocess.check_call(base + ["-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("walls", C.c_int),
                ("tau_out", C.c_double), ("tau_in", C.c_double), ("rho0", C.c_double),
                ("body_force", C.c_double * 3), ("sigma", C.c_double), ("wetting", C.c_int),
                ("A", C.c_double), ("xi", C.c_double), ("n", C.c_int), ("m", C.c_int),
                ("h_min_frac", C.c_double), ("volume_correction", C.c_int),
                ("shear_modulus", C.c_double), ("area_modulus", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        # one thread unless asked otherwise (set_threads, or ORACLE_THREADS)
        L.orc_set_threads(int(os.environ.get("ORACLE_THREADS", "1")))
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        pp = C.POINTER(Params)
        sig = {
            "orc_d3q19": (None, [ip, dp, ip]),
            "orc_feq": (None, [C.c_double, dp, dp]),
            "orc_guo_source": (None, [C.c_double, dp, dp, dp]),
            "orc_collide_cell": (None, [C.c_double, dp, dp, dp, dp]),
            "orc_psi": (C.c_double, [C.c_double]),
            "orc_spread": (None, [pp, dp, dp, C.c_int, dp]),
            "orc_interp": (None, [pp, dp, C.c_int, dp, dp]),
            "orc_wetting_A": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]),
            "orc_Pi": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]),
            "orc_membrane_forces": (C.c_int, [pp, dp, C.c_int, ip, C.c_int, dp, dp, dp]),
            "orc_membrane_elastic": (None, [pp, dp, dp, C.c_int, ip, C.c_int, dp]),
            "orc_mesh_area": (C.c_double, [dp, ip, C.c_int]),
            "orc_mesh_volume": (C.c_double, [dp, ip, C.c_int]),
            "orc_inside": (None, [pp, dp, ip, C.c_int, C.POINTER(C.c_ubyte)]),
            "orc_theta_from_height": (C.c_double, [C.c_double, C.c_double]),
            "orc_mesh_observe": (None, [dp, C.c_int, ip, C.c_int, C.c_double, C.c_double,
                                        C.c_double, C.c_double, dp]),
            "orc_create": (C.c_void_p, [pp]),
            "orc_destroy": (None, [C.c_void_p]),
            "orc_set_membrane": (C.c_int, [C.c_void_p, dp, C.c_int, ip, C.c_int]),
            "orc_set_nodes": (None, [C.c_void_p, dp]),
            "orc_get_nodes": (None, [C.c_void_p, dp]),
            "orc_set_populations": (None, [C.c_void_p, dp]),
            "orc_get_populations": (None, [C.c_void_p, dp]),
            "orc_step": (None, [C.c_void_p, C.c_int]),
            "orc_set_threads": (None, [C.c_int]),
            "orc_get_threads": (C.c_int, []),
            "orc_get_macros": (None, [C.c_void_p, dp, dp]),
            "orc_get_force_density": (None, [C.c_void_p, dp]),
            "orc_get_node_forces": (None, [C.c_void_p, dp]),
            "orc_get_tau": (None, [C.c_void_p, dp]),
            "orc_observe": (None, [C.c_void_p, C.c_double, C.c_double, dp]),
            "orc_clamped_nodes": (C.c_long, [C.c_void_p]),
            "orc_cells": (C.c_long, [C.c_void_p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def make_params(nx, ny, nz, walls=1, tau_out=1.0, tau_in=None, rho0=1.0, body_force=(0, 0, 0),
                sigma=0.0, wetting=0, A=0.0, xi=1.0, n=6, m=3, h_min_frac=0.5,
                volume_correction=0, shear_modulus=0.0, area_modulus=0.0) -> Params:
    p = Params()
    p.nx, p.ny, p.nz, p.walls = nx, ny, nz, walls
    p.tau_out = tau_out
    p.tau_in = tau_out if tau_in is None else tau_in
    p.rho0 = rho0
    p.body_force = (C.c_double * 3)(*body_force)
    p.sigma, p.wetting, p.A, p.xi, p.n, p.m = sigma, wetting, A, xi, n, m
    p.h_min_frac, p.volume_correction = h_min_frac, volume_correction
    p.shear_modulus, p.area_modulus = shear_modulus, area_modulus
    return p


def d3q19():
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    lib().orc_d3q19(_i(c), _d(w), _i(opp))
    return c, w, opp


def feq(rho, u):
    out = np.zeros(19)
    lib().orc_feq(rho, _d(f64(u)), _d(out))
    return out


def guo_source(tau, u, F):
    out = np.zeros(19)
    lib().orc_guo_source(tau, _d(f64(u)), _d(f64(F)), _d(out))
    return out


def collide_cell(tau, F, f):
    f = f64(f).copy()
    rho = np.zeros(1)
    u = np.zeros(3)
    lib().orc_collide_cell(tau, _d(f64(F)), _d(f), _d(rho), _d(u))
    return f, rho[0], u


def psi(r):
    return lib().orc_psi(float(r))


def wetting_A(sigma, theta, xi, n=6, m=3):
    return lib().orc_wetting_A(sigma, theta, xi, n, m)


def Pi(h, A, xi, n=6, m=3):
    return lib().orc_Pi(h, A, xi, n, m)


def cells_of(p: Params):
    return p.nx * p.ny * (p.nz - 2 if p.walls else p.nz)


def spread(p, xyz, phi):
    xyz, phi = f64(xyz), f64(phi)
    F = np.zeros(3 * cells_of(p))
    lib().orc_spread(C.byref(p), _d(xyz), _d(phi), len(xyz), _d(F))
    return F


def interp(p, xyz, U):
    xyz, U = f64(xyz), f64(U)
    out = np.zeros((len(xyz), 3))
    lib().orc_interp(C.byref(p), _d(xyz), len(xyz), _d(U), _d(out))
    return out


def membrane_elastic(p, xyz_ref, xyz, tri):
    """Skalak elastic forces of the mesh xyz against the reference xyz_ref."""
    xyz_ref, xyz, tri = f64(xyz_ref), f64(xyz), i32(tri)
    phi = np.zeros((len(xyz), 3))
    lib().orc_membrane_elastic(C.byref(p), _d(xyz_ref), _d(xyz), len(xyz), _i(tri), len(tri), _d(phi))
    return phi


def membrane_forces(p, xyz, tri):
    xyz, tri = f64(xyz), i32(tri)
    n = len(xyz)
    phi, fs, fp = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    clamped = lib().orc_membrane_forces(C.byref(p), _d(xyz), n, _i(tri), len(tri), _d(phi), _d(fs), _d(fp))
    return phi, fs, fp, clamped


def mesh_area(xyz, tri):
    return lib().orc_mesh_area(_d(f64(xyz)), _i(i32(tri)), len(tri))


def mesh_volume(xyz, tri):
    return lib().orc_mesh_volume(_d(f64(xyz)), _i(i32(tri)), len(tri))


def inside(p, xyz, tri):
    out = np.zeros(cells_of(p), np.uint8)
    lib().orc_inside(C.byref(p), _d(f64(xyz)), _i(i32(tri)), len(tri),
                     out.ctypes.data_as(C.POINTER(C.c_ubyte)))
    return out


def theta_from_height(ell, R):
    return lib().orc_theta_from_height(ell, R)


def mesh_observe(xyz, tri, R0, z_wall=0.5, zcut_frac=0.05, eps_flat=0.1):
    out = np.zeros(len(OBS_NAMES))
    xyz, tri = f64(xyz), i32(tri)
    lib().orc_mesh_observe(_d(xyz), len(xyz), _i(tri), len(tri), R0, z_wall, zcut_frac, eps_flat, _d(out))
    return dict(zip(OBS_NAMES, out))


class Sim:
    """The oracle's full IB-LB time step (oracle.c one_step)."""

    def __init__(self, p: Params):
        self.p = p
        self.h = lib().orc_create(C.byref(p))
        self.cells = lib().orc_cells(self.h)
        self.n_nodes = 0
        self.tri = None

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def set_membrane(self, xyz, tri):
        xyz, tri = f64(xyz), i32(tri)
        self.n_nodes = len(xyz)
        self.tri = tri
        lib().orc_set_membrane(self.h, _d(xyz), len(xyz), _i(tri), len(tri))

    def set_nodes(self, xyz):
        lib().orc_set_nodes(self.h, _d(f64(xyz)))

    def nodes(self):
        out = np.zeros((self.n_nodes, 3))
        lib().orc_get_nodes(self.h, _d(out))
        return out

    def set_populations(self, f):
        lib().orc_set_populations(self.h, _d(f64(f)))

    def populations(self):
        out = np.zeros(19 * self.cells)
        lib().orc_get_populations(self.h, _d(out))
        return out

    def step(self, n=1):
        lib().orc_step(self.h, n)

    def macros(self):
        rho = np.zeros(self.cells)
        u = np.zeros(3 * self.cells)
        lib().orc_get_macros(self.h, _d(rho), _d(u))
        return rho, u

    def force_density(self):
        out = np.zeros(3 * self.cells)
        lib().orc_get_force_density(self.h, _d(out))
        return out

    def node_forces(self):
        out = np.zeros((self.n_nodes, 3))
        lib().orc_get_node_forces(self.h, _d(out))
        return out

    def tau(self):
        out = np.zeros(self.cells)
        lib().orc_get_tau(self.h, _d(out))
        return out

    def observe(self, zcut_frac=0.05, eps_flat=0.1):
        out = np.zeros(len(OBS_NAMES))
        lib().orc_observe(self.h, zcut_frac, eps_flat, _d(out))
        return dict(zip(OBS_NAMES, out))

    def clamped(self):
        return lib().orc_clamped_nodes(self.h)


def set_threads(n: int) -> None:
    """Threads of the stream-collide loop (1 when built without OpenMP)."""
    lib().orc_set_threads(int(n))


def threads() -> int:
    return lib().orc_get_threads()
