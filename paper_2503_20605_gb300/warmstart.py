"""Learned warm start: equilibria from batched IB-LB runs, the network that
learns them, and the comparison of a warm start against the plain sphere
start.  Orchestration only: the time steps, the observables, the network's
training and inference all run in libiblb (C ABI, CUDA); the mesh profile
and the mesh deformation are the library's host functions.

Definitions (this project's; the paper uses no network):
  * a case is (theta_eq in degrees, R0, lambda); the droplet is the
    icosphere of radius R0 (level by radius), sigma = 0.01, xi =
    max(2, 0.1 R0), volume correction on, FP16 storage, in a box sized to
    hold the equilibrium cap (`case_box`).  The viscosities keep the ratio
    lambda (eq. def_lambda) with both relaxation times in [0.6, 1.5]:
    (tau_out - 1/2)(tau_in - 1/2) = 0.1, i.e. tau_out = 1/2 + sqrt(0.1 /
    lambda), tau_in = 1/2 + sqrt(0.1 lambda) -- a fixed tau_out with
    lambda = 0.1 puts tau_in next to 1/2, where the droplet breaks up;
  * the equilibrium is reached at the first observation (every `every`
    steps, at least `min_steps` in) at which the contact angle (eq. angleh
    with the volume-equivalent radius) has moved less than `tol_deg` over
    the last `window` steps;
  * the label of a case is the radial profile g(phi) = G(phi) / R0 of its
    mesh at equilibrium about the node centroid (App. B parametrisation,
    64 polar samples);
  * a warm start deforms the sphere mesh to the network's predicted profile
    (nodes keep their azimuth and share of the surface area) at the
    sphere's volume, lowest node at h = xi.

    python -m paper_2503_20605_gb300.warmstart --train 2000 --test 200
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import iblb
from . import inputs as I

SIGMA = 0.01
NU_PRODUCT = 0.1       # (tau_out - 1/2)(tau_in - 1/2)


def tau_out_for(lam):
    return 0.5 + math.sqrt(NU_PRODUCT / lam)


def cap_extent(theta_deg, R):
    """Horizontal half-width and height of the spherical cap of contact
    angle theta with the volume of a sphere of radius R."""
    c = math.cos(math.radians(theta_deg))
    rho = R * (4.0 / (2.0 - 3.0 * c + c ** 3)) ** (1.0 / 3.0)
    half = rho * math.sin(math.radians(theta_deg)) if theta_deg <= 90.0 else rho
    return half, rho * (1.0 - c)


def cap_profile(theta_deg, nphi=iblb.NPHI):
    """Profile g(phi_k) = G / R0 of an exact spherical cap with contact
    angle theta_deg and the volume of the unit sphere, about the centroid of
    its surface, at phi_k = (k + 1/2) pi / nphi: the spherical-cap start of
    Sec. III B (computed by the library, iblb_cap_profile)."""
    return iblb.iblb_cap_profile(theta_deg, nphi)


def case_box(theta_deg, R, xi):
    """Box holding both the initial sphere and the equilibrium cap with 8
    cells of margin on each side (multiples of 8; walls at Z = 0, nz - 1)."""
    half, hcap = cap_extent(theta_deg, R)
    side = max(2.0 * half, 2.0 * R) + 16.0
    n = max(48, int(math.ceil(side / 8.0)) * 8)
    h = max(2.0 * R, hcap) + xi + 12.0
    nz = max(40, int(math.ceil(h / 8.0)) * 8) + 2
    return n, n, nz


def case_spec(theta_deg, R, lam, storage="f16"):
    xi = max(2.0, 0.1 * R)
    nx, ny, nz = case_box(theta_deg, R, xi)
    return I.DropletSpec(nx, ny, nz, R, I.level_for_radius(R), SIGMA, theta_deg, xi, tau=tau_out_for(lam), lam=lam,
                         storage=storage, volume_correction=True)


def warm_mesh(spec, g):
    """Sphere mesh of the case deformed to the profile g (lowest node at
    h = xi above the wall plane z = 1/2)."""
    xyz, tri = I.icosphere(spec.level, spec.R, (0.0, 0.0, 0.0))
    q = iblb.iblb_deform_mesh(g, spec.R, xyz, tri, spec.nx / 2.0, spec.ny / 2.0, 0.5 + spec.xi)
    return q, tri


def run_to_equilibrium(cases, profiles=None, storage="f16", max_steps=40000, every=500, window=2000,
                       tol_deg=0.05, min_steps=2000, stream=0, log=None):
    """Run every case (rows of (theta_eq, R0, lambda)) in one batched context
    from the sphere, or from the deformed meshes when `profiles` (n x 64) is
    given, until each reaches equilibrium or max_steps.  Returns a dict of
    arrays: steps (equilibrium step, -1 if not reached), theta (contact
    angle then, eq. angleh with R_V), profile (n x 64 at that step),
    status (the device status of unstable cases, else 0), cells."""
    cases = np.asarray(cases, np.float64)
    n = len(cases)
    specs = [case_spec(t, R, lam, storage) for t, R, lam in cases]
    lats = [iblb.lattice_desc(s.nx, s.ny, s.nz, tau_out=s.tau, lam=s.lam, storage=storage) for s in specs]
    phys = [iblb.physics_desc(sigma=s.sigma, theta_eq_deg=s.theta_deg, xi=s.xi, volume_correction=1)
            for s in specs]
    ctx = iblb.iblb_batch_create(lats, phys, stream)
    steps = np.full(n, -1, np.int64)
    theta = np.full(n, np.nan)
    prof = np.full((n, iblb.NPHI), np.nan)
    hist = [[] for _ in range(n)]
    status = np.zeros(n, np.int64)
    try:
        for k, s in enumerate(specs):
            if profiles is None:
                xyz, tri = s.mesh()
            else:
                xyz, tri = warm_mesh(s, profiles[k])
            iblb.iblb_set_membrane(ctx, k, xyz, tri)
        done = 0
        lag = window // every
        while done < max_steps and np.any((steps < 0) & (status == 0)):
            iblb.iblb_step(ctx, every)
            done += every
            obs = iblb.iblb_observe_all(ctx)
            for k in range(n):
                if steps[k] >= 0 or status[k] != 0:
                    continue
                o = obs[k]
                status[k] = o["status"]
                if status[k] != 0:      # unstable: no equilibrium for this case
                    continue
                hist[k].append(o["theta_RV_deg"])
                if (done >= min_steps and len(hist[k]) > lag
                        and abs(hist[k][-1] - hist[k][-1 - lag]) < tol_deg):
                    steps[k] = done
                    theta[k] = o["theta_RV_deg"]
                    prof[k] = iblb.iblb_mesh_profile(iblb.iblb_get_nodes(ctx, k), specs[k].R)
            if log:
                log(f"  {done} steps: {int(np.sum(steps >= 0))}/{n} at equilibrium")
        for k in range(n):   # not converged but stable: report the last state
            if steps[k] < 0 and status[k] == 0:
                o = iblb.iblb_observe(ctx, k)
                theta[k] = o["theta_RV_deg"]
                prof[k] = iblb.iblb_mesh_profile(iblb.iblb_get_nodes(ctx, k), specs[k].R)
    finally:
        iblb.iblb_destroy(ctx)
    return {"steps": steps, "theta": theta, "profile": prof, "status": status,
            "cells": np.array([s.nx * s.ny * (s.nz - 2) for s in specs])}


def generate(cases, batch=64, **kw):
    """Equilibria of many cases, `batch` droplets per context."""
    out = []
    for b0 in range(0, len(cases), batch):
        out.append(run_to_equilibrium(cases[b0:b0 + batch], **kw))
    return {k: np.concatenate([o[k] for o in out]) for k in out[0]}


def train(x, y, epochs=2000, batch=256, lr=1e-3, seed=0, init_seed=0, stream=0):
    """Train the network on (x, y); returns (parameters, loss per epoch)."""
    m = iblb.iblb_mlp_create(I.mlp_init(init_seed), batch, stream)
    try:
        losses = iblb.iblb_mlp_train(m, x, y, epochs, batch, lr, seed)
        return iblb.iblb_mlp_get_params(m), losses
    finally:
        iblb.iblb_mlp_destroy(m)


PARAMS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "warmstart_mlp_params.npy")


def load_params(path=PARAMS_PATH):
    """The trained network's parameters shipped with the package (made by
    this module's command line; provenance in the .json beside them)."""
    return np.load(path).astype(np.float32)


def predict(params, x, stream=0):
    m = iblb.iblb_mlp_create(params, 256, stream)
    try:
        return iblb.iblb_mlp_predict(m, x)
    finally:
        iblb.iblb_mlp_destroy(m)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--max-steps", type=int, default=40000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=2000)
    ap.add_argument("--mlp-batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default="warmstart_results")
    ap.add_argument("--train-data", default=None,
                    help="train_data.npz of an earlier run: train on its equilibria instead of generating them")
    args = ap.parse_args(argv)
    import torch
    torch.cuda.init()
    stream = torch.cuda.current_stream().cuda_stream
    os.makedirs(args.out, exist_ok=True)
    log = lambda s: print(s, flush=True)
    t0 = time.time()
    xtr = I.warmstart_cases(args.train, 1)
    xte = I.warmstart_cases(args.test, 2)
    if args.train_data:
        with np.load(args.train_data) as z:
            tr = {k: z[k] for k in z.files if k != "x"}
            xtr = z["x"]
        args.train = len(xtr)
        ok = tr["steps"] >= 0
        log(f"{ok.sum()} of {len(xtr)} training equilibria from {args.train_data}")
    else:
        log(f"generating {args.train} training equilibria")
        tr = generate(xtr, batch=args.batch, max_steps=args.max_steps, stream=stream, log=log)
        ok = tr["steps"] >= 0
        log(f"  {ok.sum()} converged ({time.time() - t0:.0f} s)")
        np.savez(os.path.join(args.out, "train_data.npz"), x=xtr, **tr)
    params, losses = train(xtr[ok], tr["profile"][ok], epochs=args.epochs, batch=args.mlp_batch, lr=args.lr,
                           stream=stream)
    log(f"trained: loss {losses[0]:.3e} -> {losses[-1]:.3e} ({time.time() - t0:.0f} s)")
    g = predict(params, xte, stream)
    log("held-out cases from the sphere")
    sph = generate(xte, batch=args.batch, max_steps=args.max_steps, stream=stream, log=log)
    log("held-out cases from the warm start")
    warm = generate(xte, batch=args.batch, max_steps=args.max_steps, profiles=g, stream=stream, log=log)
    both = (sph["steps"] >= 0) & (warm["steps"] >= 0)
    res = {
        "train_cases": int(args.train), "train_converged": int(ok.sum()), "test_cases": int(args.test),
        "both_converged": int(both.sum()),
        "steps_sphere_mean": float(sph["steps"][both].mean()), "steps_warm_mean": float(warm["steps"][both].mean()),
        "steps_sphere_median": float(np.median(sph["steps"][both])),
        "steps_warm_median": float(np.median(warm["steps"][both])),
        "dtheta_warm_vs_sphere_mean_deg": float(np.mean(np.abs(warm["theta"][both] - sph["theta"][both]))),
        "dtheta_warm_vs_sphere_max_deg": float(np.max(np.abs(warm["theta"][both] - sph["theta"][both]))),
        "profile_rms_pred_vs_sphere_eq": float(np.sqrt(np.mean((g[both] - sph["profile"][both]) ** 2))),
        "final_loss": float(losses[-1]), "seconds": time.time() - t0,
    }
    np.save(os.path.join(args.out, "warmstart_mlp_params.npy"), params)
    np.savez(os.path.join(args.out, "warmstart.npz"), xtr=xtr, ytr=tr["profile"], steps_tr=tr["steps"], xte=xte,
             params=params, losses=losses, g=g, sph_steps=sph["steps"], warm_steps=warm["steps"],
             sph_theta=sph["theta"], warm_theta=warm["theta"], sph_profile=sph["profile"])
    print(json.dumps(res))
    return res


if __name__ == "__main__":
    sys.exit(0 if main() else 1)
