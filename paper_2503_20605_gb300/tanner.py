"""Late-stage spreading from a spherical-cap start (Sec. III B): the viscous
regime where Tanner's law r_c ~ t^(1/10) is expected before the droplet
settles.  Orchestration only: the initial cap comes from the library's
iblb_cap_profile and iblb_deform_mesh, the time steps and the observables
run in libiblb (C ABI, CUDA).

Set-up (the paper gives xi = 3, R0 = 90 .. 150, small theta_eq and a
spherical-cap start that skips the inertial stage; the rest is this
project's reading):
  * an icosphere of radius R0 deformed to the exact spherical cap of angle
    theta0 > theta_eq (default 90 degrees) at the sphere's volume, lowest
    node at h = xi above the wall plane;
  * D3Q19, tau = 1 inside and out (lambda = 1), sigma = 0.01, walls at
    Z = 0 and nz - 1, volume correction on, FP16 offsets;
  * a box wide enough for the equilibrium cap of angle theta_eq;
  * the contact radius by protocol (i) with the plane at the minimum of
    Pi(h), h* = xi (n/m)^(1/(n-m)) = 2^(1/3) xi; time in units of the
    viscous time t* = mu R0 / sigma (mu = rho (tau - 1/2) / 3).

    python -m paper_2503_20605_gb300.tanner --R0 60 --steps 200000
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from . import iblb
from . import inputs as I

SIGMA = 0.01
TAU = 1.0


def cap_box(theta_eq_deg, theta0_deg, R0, xi):
    """Box holding the equilibrium cap of angle theta_eq (its footprint) and
    the initial cap of angle theta0 (its height), 16 cells of margin around
    the footprint; sides multiples of 16, walls at Z = 0 and nz - 1."""
    def extent(th):
        c = math.cos(math.radians(th))
        rho = R0 * (4.0 / (2.0 - 3.0 * c + c ** 3)) ** (1.0 / 3.0)
        half = rho * math.sin(math.radians(th)) if th <= 90.0 else rho
        return half, rho * (1.0 - c)
    half_eq, _ = extent(theta_eq_deg)
    half0, h0 = extent(theta0_deg)
    side = 2.0 * max(half_eq, half0) + 32.0
    n = int(math.ceil(side / 16.0)) * 16
    nz = int(math.ceil((h0 + xi + 12.0) / 8.0)) * 8 + 2
    return n, n, nz


def cap_mesh(R0, level, theta0_deg, nx, ny, xi):
    """The icosphere of radius R0 deformed to the spherical cap of angle
    theta0 (same volume), centred in x and y, lowest node at h = xi."""
    xyz, tri = I.icosphere(level, R0, (0.0, 0.0, 0.0))
    g = iblb.iblb_cap_profile(theta0_deg)
    q = iblb.iblb_deform_mesh(g, R0, xyz, tri, nx / 2.0, ny / 2.0, 0.5 + xi)
    return q, tri


def run(R0=60.0, theta_eq_deg=22.5, theta0_deg=90.0, xi=3.0, level=7, steps=200000, every=1000,
        storage="f16", stream=0, log=None):
    """Run the cap start for `steps` steps, observing every `every` steps.
    Returns a dict with the times (steps), t / t*, r_c / R0 (protocol (i)),
    the contact angle (eq. angleh with R_V), V / V0, the device status and
    the set-up."""
    nx, ny, nz = cap_box(theta_eq_deg, theta0_deg, R0, xi)
    lat = iblb.lattice_desc(nx, ny, nz, tau_out=TAU, storage=storage)
    phys = iblb.physics_desc(sigma=SIGMA, theta_eq_deg=theta_eq_deg, xi=xi, volume_correction=1)
    xyz, tri = cap_mesh(R0, level, theta0_deg, nx, ny, xi)
    t_star = (TAU - 0.5) / 3.0 * R0 / SIGMA
    zcut_frac = xi * 2.0 ** (1.0 / 3.0) / R0
    ctx = iblb.iblb_create(lat, phys, stream)
    out = {"R0": R0, "theta_eq_deg": theta_eq_deg, "theta0_deg": theta0_deg, "xi": xi, "level": level,
           "box": [nx, ny, nz], "nodes": len(xyz), "faces": len(tri), "t_star": t_star, "storage": storage,
           "step": [], "t": [], "rc": [], "theta_RV_deg": [], "volume_ratio": [], "status": 0}
    t0 = time.perf_counter()
    try:
        iblb.iblb_set_membrane(ctx, 0, xyz, tri)
        V0 = iblb.iblb_observe(ctx, 0, zcut_frac, 0.1)["volume"]
        done = 0
        while done < steps:
            n = min(every, steps - done)
            iblb.iblb_step(ctx, n)
            done += n
            o = iblb.iblb_observe(ctx, 0, zcut_frac, 0.1)
            out["step"].append(done)
            out["t"].append(done / t_star)
            out["rc"].append(o["rc_cut"] / R0)
            out["theta_RV_deg"].append(o["theta_RV_deg"])
            out["volume_ratio"].append(o["volume"] / V0)
            if o["status"]:
                out["status"] = o["status"]
                break
            if log:
                log(f"step {done}: t/t* {done / t_star:.2f} r_c/R0 {o['rc_cut'] / R0:.4f} "
                    f"theta {o['theta_RV_deg']:.2f}")
    finally:
        iblb.iblb_destroy(ctx)
    out["seconds"] = time.perf_counter() - t0
    return out


def local_exponents(t, r, width=0.3):
    """d ln r / d ln t by a least-squares line over windows of `width` in
    log10 t, centred at each sample with a full window."""
    lt, lr = np.log10(np.asarray(t)), np.log10(np.asarray(r))
    res = []
    for i in range(len(lt)):
        sel = np.abs(lt - lt[i]) <= width / 2
        if lt[i] - width / 2 < lt[0] or lt[i] + width / 2 > lt[-1] or sel.sum() < 3:
            continue
        res.append((10 ** lt[i], np.polyfit(lt[sel], lr[sel], 1)[0]))
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--R0", type=float, default=60.0)
    ap.add_argument("--theta-eq", type=float, default=22.5)
    ap.add_argument("--theta0", type=float, default=90.0)
    ap.add_argument("--xi", type=float, default=3.0)
    ap.add_argument("--level", type=int, default=7)
    ap.add_argument("--steps", type=int, default=200000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--storage", default="f16")
    ap.add_argument("--out", default=None, help="write the run as JSON here")
    a = ap.parse_args(argv)
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    res = run(a.R0, a.theta_eq, a.theta0, a.xi, a.level, a.steps, a.every, a.storage, stream,
              log=lambda s: print(s, file=sys.stderr, flush=True))
    res["local_exponents"] = local_exponents(res["t"], res["rc"])
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f)
    for tt, k in res["local_exponents"][::5]:
        print(f"t/t* {tt:8.2f}  d ln r_c / d ln t {k:.3f}")
    print(json.dumps({k: res[k] for k in ("box", "nodes", "faces", "t_star", "status", "seconds")}))


if __name__ == "__main__":
    main()
