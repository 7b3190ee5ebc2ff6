"""Helpers shared by the GPU tests: build a CUDA context and an oracle
simulation from the same seeded inputs."""
import math

import numpy as np

import oracle.oracle as O
from paper_2503_20605_gb300 import iblb


def stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def gpu_ctx(nx, ny, nz, tau=1.0, lam=1.0, storage="f32", walls=1, body_force=(0, 0, 0), sigma=0.0,
            theta=None, xi=2.0, h_min_frac=0.5, volume_correction=0, mesh=None, shear_modulus=0.0,
            area_modulus=0.0):
    lat = iblb.lattice_desc(nx, ny, nz, tau_out=tau, lam=lam, storage=storage, walls=walls, body_force=body_force)
    phys = iblb.physics_desc(sigma=sigma, theta_eq_deg=theta, xi=xi, h_min_frac=h_min_frac,
                             volume_correction=volume_correction, shear_modulus=shear_modulus,
                             area_modulus=area_modulus)
    ctx = iblb.iblb_create(lat, phys, stream())
    if mesh is not None:
        iblb.iblb_set_membrane(ctx, 0, mesh[0], mesh[1])
    return ctx


def oracle_sim(nx, ny, nz, tau=1.0, lam=1.0, walls=1, body_force=(0, 0, 0), sigma=0.0, theta=None, xi=2.0,
               h_min_frac=0.5, volume_correction=0, mesh=None, shear_modulus=0.0, area_modulus=0.0):
    tau_in = 0.5 + lam * (tau - 0.5)
    A = O.wetting_A(sigma, math.radians(theta), xi) if theta is not None else 0.0
    p = O.make_params(nx, ny, nz, walls=walls, tau_out=tau, tau_in=tau_in, body_force=body_force, sigma=sigma,
                      wetting=int(theta is not None), A=A, xi=xi, h_min_frac=h_min_frac,
                      volume_correction=volume_correction, shear_modulus=shear_modulus,
                      area_modulus=area_modulus)
    s = O.Sim(p)
    if mesh is not None:
        s.set_membrane(mesh[0], mesh[1])
    return s


def pair(**kw):
    return gpu_ctx(**kw), oracle_sim(**{k: v for k, v in kw.items() if k != "storage"})


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
