"""ctypes binding of libiblb (include/iblb.h) with the same function names.

Argument marshalling only: every step of the IB-LB time step runs in the
CUDA library.  Functions take numpy arrays (host) or integer device pointers
where the C ABI takes device pointers, and raise IblbError on a non-zero
status.  The first call loads libiblb.so and raises OSError if it is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libiblb.so")

IBLB_OK = 0
IBLB_E_ARG, IBLB_E_MESH, IBLB_E_NOMEM, IBLB_E_CUDA = -1, -2, -3, -4
IBLB_E_UNSTABLE, IBLB_E_TIMEOUT, IBLB_E_STATE, IBLB_E_IO, IBLB_E_OVERFLOW = -5, -6, -7, -8, -9
IBLB_STORE_F32, IBLB_STORE_F16, IBLB_STORE_BF16 = 0, 1, 2
STORAGE = {"f32": IBLB_STORE_F32, "f16": IBLB_STORE_F16, "bf16": IBLB_STORE_BF16}
IBLB_WET_OFF, IBLB_WET_THETA, IBLB_WET_RAW = 0, 1, 2
IBLB_PH_FORCES, IBLB_PH_SPREAD, IBLB_PH_INOUT, IBLB_PH_LB, IBLB_PH_ADVECT, IBLB_PH_REDUCE = range(6)
IBLB_NPHASE = 6
IBLB_TRACE_FORCE, IBLB_TRACE_SPREAD, IBLB_TRACE_LB, IBLB_TRACE_INTERP, IBLB_TRACE_VC = range(5)
IBLB_TRACE_KERNELS = 5
PHASE_NAMES = ["forces", "spread", "inout", "lb", "advect", "reduce"]
IBLB_OPT_GRAPHS, IBLB_OPT_PROFILE, IBLB_OPT_LB_BLOCKS_PER_SM, IBLB_OPT_LB_ROW_MULT, IBLB_OPT_LB_STAGES = 0, 1, 2, 3, 4
IBLB_OPT_FUSED_IB, IBLB_OPT_IB_BLOCKS_PER_SM, IBLB_OPT_SPLIT_LB, IBLB_OPT_LB_FAR_BLOCKS_PER_SM = 5, 6, 7, 8
IBLB_OPT_PDL, IBLB_OPT_LB_GROUP_CELLS, IBLB_OPT_GRAPH_CHUNK = 9, 10, 11

CODE_NAMES = {0: "IBLB_OK", -1: "IBLB_E_ARG", -2: "IBLB_E_MESH", -3: "IBLB_E_NOMEM", -4: "IBLB_E_CUDA",
              -5: "IBLB_E_UNSTABLE", -6: "IBLB_E_TIMEOUT", -7: "IBLB_E_STATE", -8: "IBLB_E_IO",
              -9: "IBLB_E_OVERFLOW"}


class IblbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{CODE_NAMES.get(code, code)}: {msg}")
        self.code = code


class LatticeDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("walls", C.c_int),
                ("tau_out", C.c_double), ("lambda_", C.c_double), ("rho0", C.c_double),
                ("storage", C.c_int), ("body_force", C.c_double * 3)]


class PhysicsDesc(C.Structure):
    _fields_ = [("sigma", C.c_double), ("wetting", C.c_int), ("theta_eq_deg", C.c_double),
                ("A", C.c_double), ("xi", C.c_double), ("n", C.c_int), ("m", C.c_int),
                ("h_min_frac", C.c_double), ("volume_correction", C.c_int),
                ("shear_modulus", C.c_double), ("area_modulus", C.c_double)]


class Obs(C.Structure):
    _fields_ = [("mass", C.c_double), ("volume", C.c_double), ("area", C.c_double),
                ("centroid", C.c_double * 3), ("zmin", C.c_double), ("zmax", C.c_double),
                ("theta_R0_deg", C.c_double), ("theta_RV_deg", C.c_double), ("rc_cut", C.c_double),
                ("rc_flat", C.c_double), ("n_cut", C.c_double), ("chi_flat", C.c_double),
                ("status", C.c_int), ("clamped", C.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "centroid"}
        d["cx"], d["cy"], d["cz"] = tuple(self.centroid)
        return d


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_SIGS = {
    "iblb_version": (C.c_char_p, []),
    "iblb_selftest_wait_timeout": (C.c_int, [C.c_longlong, _P]),
    "iblb_last_error": (C.c_char_p, [_P]),
    "iblb_wetting_A": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _D]),
    "iblb_create": (C.c_int, [C.POINTER(LatticeDesc), C.POINTER(PhysicsDesc), _P, C.POINTER(_P)]),
    "iblb_batch_create": (C.c_int, [C.c_int, C.POINTER(LatticeDesc), C.POINTER(PhysicsDesc), _P,
                                    C.POINTER(_P)]),
    "iblb_destroy": (None, [_P]),
    "iblb_info": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int),
                            C.POINTER(C.c_int)]),
    "iblb_set_membrane": (C.c_int, [_P, C.c_int, _D, C.c_int, _I32, C.c_int]),
    "iblb_check_mesh": (C.c_int, [_D, C.c_int, _I32, C.c_int, _D]),
    "iblb_set_nodes": (C.c_int, [_P, C.c_int, _D]),
    "iblb_get_nodes": (C.c_int, [_P, C.c_int, _D]),
    "iblb_set_populations": (C.c_int, [_P, C.c_int, _D]),
    "iblb_get_populations": (C.c_int, [_P, C.c_int, _D]),
    "iblb_get_macros": (C.c_int, [_P, C.c_int, _D, _D]),
    "iblb_compute_forces": (C.c_int, [_P]),
    "iblb_get_node_forces": (C.c_int, [_P, C.c_int, _D]),
    "iblb_get_force_density": (C.c_int, [_P, C.c_int, _D]),
    "iblb_get_inside": (C.c_int, [_P, C.c_int, C.POINTER(C.c_uint8)]),
    "iblb_step": (C.c_int, [_P, C.c_int]),
    "iblb_sync": (C.c_int, [_P]),
    "iblb_trace_step": (C.c_int, [_P, _D]),
    "iblb_observe": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.POINTER(Obs)]),
    "iblb_observe_all": (C.c_int, [_P, C.c_double, C.c_double, C.POINTER(Obs)]),
    "iblb_set_option": (C.c_int, [_P, C.c_int, C.c_int]),
    "iblb_get_profile": (C.c_int, [_P, _D, _D, C.POINTER(C.c_int64)]),
    "iblb_reset_profile": (C.c_int, [_P]),
    "iblb_autotune": (C.c_int, [_P, C.c_char_p]),
    "iblb_save": (C.c_int, [_P, C.c_char_p]),
    "iblb_load": (C.c_int, [_P, C.c_char_p]),
    "iblb_mesh_observe_dev": (C.c_int, [_P, C.c_int, _P, C.c_int, C.c_double, C.c_double, C.c_double, _P, _D]),
    "iblb_mesh_observe_dev_noalloc": (C.c_int, [_P, C.c_int, _P, C.c_int, C.c_double, C.c_double, C.c_double, _P,
                                                _D]),
    "iblb_mesh_profile": (C.c_int, [_D, C.c_int, C.c_double, C.c_int, _D]),
    "iblb_deform_mesh": (C.c_int, [_D, C.c_int, C.c_double, _D, C.c_int, _I32, C.c_int, C.c_double, C.c_double,
                                   C.c_double, _D]),
    "iblb_warmstart_last_error": (C.c_char_p, []),
    "iblb_cap_profile": (C.c_int, [C.c_double, C.c_int, _D]),
    "iblb_mlp_param_count": (C.c_int64, []),
    "iblb_mlp_create": (C.c_int, [C.POINTER(C.c_float), C.c_int64, C.c_int, _P, C.POINTER(_P)]),
    "iblb_mlp_destroy": (None, [_P]),
    "iblb_mlp_last_error": (C.c_char_p, [_P]),
    "iblb_mlp_get_params": (C.c_int, [_P, C.POINTER(C.c_float), C.c_int64]),
    "iblb_mlp_predict": (C.c_int, [_P, _D, C.c_int, _D]),
    "iblb_mlp_grad": (C.c_int, [_P, _D, _D, C.c_int, _D, _D]),
    "iblb_mlp_train": (C.c_int, [_P, _D, _D, C.c_int, C.c_int, C.c_int, C.c_double, C.c_uint64, _D]),
}

_lib = None


def lib():
    """Load libiblb.so (raises OSError if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: run paper_2503_20605_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _check(ctx, rc):
    if rc != IBLB_OK:
        msg = lib().iblb_last_error(ctx)
        raise IblbError(rc, msg.decode() if msg else "")
    return rc


def iblb_version():
    return lib().iblb_version().decode()


def iblb_wetting_A(sigma, theta_eq_deg, xi, n=6, m=3):
    A = C.c_double()
    _check(None, lib().iblb_wetting_A(sigma, theta_eq_deg, xi, n, m, C.byref(A)))
    return A.value


def lattice_desc(nx, ny, nz, tau_out=1.0, lam=1.0, rho0=1.0, storage="f32", walls=1, body_force=(0, 0, 0)):
    d = LatticeDesc()
    d.nx, d.ny, d.nz, d.walls = nx, ny, nz, walls
    d.tau_out, d.lambda_, d.rho0 = tau_out, lam, rho0
    d.storage = STORAGE[storage] if isinstance(storage, str) else storage
    d.body_force = (C.c_double * 3)(*body_force)
    return d


def physics_desc(sigma=0.0, theta_eq_deg=None, A=None, xi=2.0, n=6, m=3, h_min_frac=0.5, volume_correction=0,
                 shear_modulus=0.0, area_modulus=0.0):
    p = PhysicsDesc()
    p.sigma, p.xi, p.n, p.m, p.h_min_frac = sigma, xi, n, m, h_min_frac
    p.volume_correction = int(volume_correction)
    p.shear_modulus, p.area_modulus = shear_modulus, area_modulus
    if theta_eq_deg is not None:
        p.wetting, p.theta_eq_deg = IBLB_WET_THETA, theta_eq_deg
    elif A is not None:
        p.wetting, p.A = IBLB_WET_RAW, A
    else:
        p.wetting = IBLB_WET_OFF
    return p


def iblb_create(lat: LatticeDesc, phys: PhysicsDesc, stream=0):
    h = _P()
    _check(None, lib().iblb_create(C.byref(lat), C.byref(phys), _P(stream), C.byref(h)))
    return h


def iblb_batch_create(lats, physs, stream=0):
    n = len(lats)
    la = (LatticeDesc * n)(*lats)
    pa = (PhysicsDesc * n)(*physs)
    h = _P()
    _check(None, lib().iblb_batch_create(n, la, pa, _P(stream), C.byref(h)))
    return h


def iblb_destroy(ctx):
    lib().iblb_destroy(ctx)


def iblb_info(ctx, k=0):
    nd, cells, nn, nt = C.c_int(), C.c_int64(), C.c_int(), C.c_int()
    _check(ctx, lib().iblb_info(ctx, k, C.byref(nd), C.byref(cells), C.byref(nn), C.byref(nt)))
    return dict(n_drops=nd.value, cells=cells.value, n_nodes=nn.value, n_tri=nt.value)


def iblb_set_membrane(ctx, k, xyz, tri):
    xyz = _f64(xyz)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    _check(ctx, lib().iblb_set_membrane(ctx, k, _d(xyz), xyz.size // 3, tri.ctypes.data_as(_I32), tri.size // 3))


def iblb_check_mesh(xyz, tri):
    """Host-only mesh check (no GPU); returns the enclosed volume."""
    xyz = _f64(xyz)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    V = C.c_double()
    _check(None, lib().iblb_check_mesh(_d(xyz), xyz.size // 3, tri.ctypes.data_as(_I32), tri.size // 3,
                                       C.byref(V)))
    return V.value


def iblb_set_nodes(ctx, k, xyz):
    xyz = _f64(xyz)
    _check(ctx, lib().iblb_set_nodes(ctx, k, _d(xyz)))


def iblb_get_nodes(ctx, k, out=None):
    n = iblb_info(ctx, k)["n_nodes"]
    out = np.empty((n, 3)) if out is None else out
    _check(ctx, lib().iblb_get_nodes(ctx, k, _d(out)))
    return out


def iblb_set_populations(ctx, k, f):
    cells = iblb_info(ctx, k)["cells"]
    f = _f64(f, 19 * cells)
    _check(ctx, lib().iblb_set_populations(ctx, k, _d(f)))


def iblb_get_populations(ctx, k):
    cells = iblb_info(ctx, k)["cells"]
    out = np.empty(19 * cells)
    _check(ctx, lib().iblb_get_populations(ctx, k, _d(out)))
    return out


def iblb_get_macros(ctx, k):
    cells = iblb_info(ctx, k)["cells"]
    rho, u = np.empty(cells), np.empty(3 * cells)
    _check(ctx, lib().iblb_get_macros(ctx, k, _d(rho), _d(u)))
    return rho, u


def iblb_compute_forces(ctx):
    _check(ctx, lib().iblb_compute_forces(ctx))


def iblb_get_node_forces(ctx, k):
    n = iblb_info(ctx, k)["n_nodes"]
    out = np.empty((n, 3))
    _check(ctx, lib().iblb_get_node_forces(ctx, k, _d(out)))
    return out


def iblb_get_force_density(ctx, k):
    cells = iblb_info(ctx, k)["cells"]
    out = np.empty(3 * cells)
    _check(ctx, lib().iblb_get_force_density(ctx, k, _d(out)))
    return out


def iblb_get_inside(ctx, k):
    cells = iblb_info(ctx, k)["cells"]
    out = np.empty(cells, np.uint8)
    _check(ctx, lib().iblb_get_inside(ctx, k, out.ctypes.data_as(C.POINTER(C.c_uint8))))
    return out


def iblb_step(ctx, nsteps=1):
    _check(ctx, lib().iblb_step(ctx, nsteps))


def iblb_sync(ctx):
    _check(ctx, lib().iblb_sync(ctx))


TRACE_KERNELS = ("force", "spread", "lb", "interp", "vc")


def iblb_trace_step(ctx):
    """One traced step: per kernel (force, spread, lb, interp, vc) a dict of
    first_start_us, median_start_us, last_start_us (warps past their wait on
    the previous kernel), end_us (the next kernel's first start, after this
    one's last exit), all from the step's earliest stamp, and warps; None for
    a kernel that did not run."""
    out = (C.c_double * (IBLB_TRACE_KERNELS * 5))()
    _check(ctx, lib().iblb_trace_step(ctx, out))
    res = {}
    for k, name in enumerate(TRACE_KERNELS):
        o = list(out[5 * k:5 * k + 5])
        res[name] = None if o[4] == 0 else {"first_start_us": o[0], "median_start_us": o[1],
                                            "last_start_us": o[2], "end_us": o[3], "warps": int(o[4])}
    return res


def iblb_observe(ctx, k=0, zcut_frac=0.05, eps_flat=0.1):
    o = Obs()
    _check(ctx, lib().iblb_observe(ctx, k, zcut_frac, eps_flat, C.byref(o)))
    return o.as_dict()


def iblb_observe_all(ctx, zcut_frac=0.05, eps_flat=0.1):
    n = iblb_info(ctx, 0)["n_drops"]
    arr = (Obs * n)()
    _check(ctx, lib().iblb_observe_all(ctx, zcut_frac, eps_flat, arr))
    return [o.as_dict() for o in arr]


def iblb_set_option(ctx, option, value):
    _check(ctx, lib().iblb_set_option(ctx, option, int(value)))


def iblb_get_profile(ctx):
    ph = (C.c_double * IBLB_NPHASE)()
    step, steps = C.c_double(), C.c_int64()
    _check(ctx, lib().iblb_get_profile(ctx, ph, C.byref(step), C.byref(steps)))
    return dict(zip(PHASE_NAMES, list(ph))), step.value, steps.value


def iblb_reset_profile(ctx):
    _check(ctx, lib().iblb_reset_profile(ctx))


def iblb_autotune(ctx, cache_path=None):
    _check(ctx, lib().iblb_autotune(ctx, cache_path.encode() if cache_path else None))


def iblb_save(ctx, path):
    _check(ctx, lib().iblb_save(ctx, str(path).encode()))


def iblb_load(ctx, path):
    _check(ctx, lib().iblb_load(ctx, str(path).encode()))


def iblb_mesh_observe_dev(d_xyz, n_nodes, d_tri, n_tri, R0, zcut_frac=0.05, eps_flat=0.1, stream=0):
    """d_xyz, d_tri: device pointers (ints, e.g. tensor.data_ptr())."""
    out = np.empty(13)
    _check(None, lib().iblb_mesh_observe_dev(_P(d_xyz), n_nodes, _P(d_tri), n_tri, R0, zcut_frac, eps_flat,
                                             _P(stream), _d(out)))
    return out


def iblb_mesh_observe_dev_noalloc(d_xyz, n_nodes, d_tri, n_tri, R0, zcut_frac=0.05, eps_flat=0.1, stream=0):
    """As iblb_mesh_observe_dev, with the scratch in a fixed device array (no allocation)."""
    out = np.empty(13)
    _check(None, lib().iblb_mesh_observe_dev_noalloc(_P(d_xyz), n_nodes, _P(d_tri), n_tri, R0, zcut_frac,
                                                     eps_flat, _P(stream), _d(out)))
    return out


# ------------------------------------------------------------ learned warm start
NPHI = 64


def _wcheck(rc):
    if rc != IBLB_OK:
        msg = lib().iblb_warmstart_last_error()
        raise IblbError(rc, msg.decode() if msg else "")


def _mcheck(m, rc):
    if rc != IBLB_OK:
        msg = lib().iblb_mlp_last_error(m)
        raise IblbError(rc, msg.decode() if msg else "")


def iblb_mesh_profile(xyz, R0, nphi=NPHI):
    xyz = _f64(xyz)
    g = np.empty(nphi)
    _wcheck(lib().iblb_mesh_profile(_d(xyz), xyz.size // 3, R0, nphi, _d(g)))
    return g


def iblb_deform_mesh(g, R0, xyz, tri, cx, cy, z_bottom):
    g = _f64(g)
    xyz = _f64(xyz)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    out = np.empty_like(xyz)
    _wcheck(lib().iblb_deform_mesh(_d(g), g.size, R0, _d(xyz), xyz.size // 3, tri.ctypes.data_as(_I32),
                                   tri.size // 3, cx, cy, z_bottom, _d(out)))
    return out


def iblb_cap_profile(theta_eq_deg, nphi=None):
    n = NPHI if nphi is None else int(nphi)
    out = np.empty(n)
    _wcheck(lib().iblb_cap_profile(float(theta_eq_deg), n, _d(out)))
    return out


def iblb_mlp_param_count():
    return int(lib().iblb_mlp_param_count())


def iblb_mlp_create(params, max_batch=256, stream=0):
    p = np.ascontiguousarray(params, dtype=np.float32)
    h = _P()
    _mcheck(None, lib().iblb_mlp_create(p.ctypes.data_as(C.POINTER(C.c_float)), p.size, max_batch, _P(stream),
                                        C.byref(h)))
    return h


def iblb_mlp_destroy(m):
    lib().iblb_mlp_destroy(m)


def iblb_mlp_get_params(m):
    out = np.empty(iblb_mlp_param_count(), dtype=np.float32)
    _mcheck(m, lib().iblb_mlp_get_params(m, out.ctypes.data_as(C.POINTER(C.c_float)), out.size))
    return out


def iblb_mlp_predict(m, x):
    x = _f64(x)
    S = x.size // 3
    y = np.empty((S, NPHI))
    _mcheck(m, lib().iblb_mlp_predict(m, _d(x), S, _d(y)))
    return y


def iblb_mlp_grad(m, x, y):
    x, y = _f64(x), _f64(y)
    S = x.size // 3
    g = np.empty(iblb_mlp_param_count())
    loss = C.c_double()
    _mcheck(m, lib().iblb_mlp_grad(m, _d(x), _d(y), S, _d(g), C.byref(loss)))
    return g, loss.value


def iblb_mlp_train(m, x, y, epochs, batch=256, lr=1e-3, seed=0):
    x, y = _f64(x), _f64(y)
    S = x.size // 3
    losses = np.zeros(max(epochs, 1))
    _mcheck(m, lib().iblb_mlp_train(m, _d(x), _d(y), S, epochs, batch, lr, seed, _d(losses)))
    return losses[:epochs]


def iblb_selftest_wait_timeout(cycles, stream=0):
    """Run the bounded mbarrier wait on a barrier that never completes;
    returns the status code (IBLB_E_TIMEOUT is the expected outcome)."""
    return lib().iblb_selftest_wait_timeout(int(cycles), _P(stream))
