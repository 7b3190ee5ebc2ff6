"""Writes statics64_oracle.txt: the FP64 oracle's trajectory of the
half-scale statics case (64^3 box, tau = 1, L4 icosphere of R = 12,
sigma = 0.005, xi = 2, wetting from theta_eq by Eq. A_choice, wall plane at
z = 0.5 per Sec. III, no volume correction) for theta_eq in {30, 60, 90,
120, 150} degrees, observed every 1000 steps up to 20000 (the step count
of the 128^3 statics sweep).  The contact angle follows Eq. angleh with
the initial radius R0 and with the current volume-equivalent radius.  Only oracle/ and the seeded input module are
used; the five runs go to five processes (spawned) and take about 40 min.

    python tests/golden/make_statics64.py
"""
import math
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

ANGLES = (30.0, 60.0, 90.0, 120.0, 150.0)
STEPS, EVERY = 20000, 1000
COLS = ("volume", "area", "zmin", "zmax", "theta_R0", "theta_RV", "rc_cut", "rc_flat", "mass")


def run(theta):
    import oracle.oracle as O
    from paper_2503_20605_gb300 import inputs as I
    w = I.workload_statics_64(theta)
    xyz, tri = w.mesh()
    A = O.wetting_A(w.sigma, math.radians(w.theta_deg), w.xi)
    p = O.make_params(w.nx, w.ny, w.nz, walls=1, tau_out=w.tau, tau_in=w.tau_in, sigma=w.sigma, wetting=1, A=A,
                      xi=w.xi, volume_correction=0)
    s = O.Sim(p)
    s.set_membrane(xyz, tri)
    rows = [(theta, 0, s.observe(0.05, 0.1))]
    for k in range(STEPS // EVERY):
        s.step(EVERY)
        rows.append((theta, (k + 1) * EVERY, s.observe(0.05, 0.1)))
    return rows


def main():
    import oracle.oracle as O
    O.build()
    with mp.get_context("spawn").Pool(len(ANGLES)) as pool:
        res = pool.map(run, ANGLES)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "statics64_oracle.txt")
    with open(out, "w") as f:
        f.write("# FP64 oracle, half-scale statics case (Sec. III statics; contact angle by Eq. angleh):\n")
        f.write("# 64^3, tau=1, L4 icosphere R=12 with lowest node at h=xi, sigma=0.005, xi=2, no volume\n")
        f.write("# correction; observables with z_cut = 0.05 R0, eps_flat = 0.1.  Written by make_statics64.py.\n")
        f.write("# theta_eq step " + " ".join(COLS) + "\n")
        for rows in res:
            for th, st, o in rows:
                f.write(f"{th:g} {st} " + " ".join(repr(float(o[c])) for c in COLS) + "\n")


if __name__ == "__main__":
    main()
