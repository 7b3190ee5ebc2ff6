"""Early spreading dynamics (Sec. III B) through the C ABI.

The inertial regime needs a small Ohnesorge number (the paper takes a larger
R0 for the dynamics to lower it).  The run here is the spreading box of the
benchmark -- 256 x 256 x 128, lambda = 10, an L6 icosphere (40 962 nodes) of
R0 = 40 released with its lowest node at h = xi = 2, theta_eq = 20 degrees,
sigma = 0.005, BF16 offsets -- with the outer relaxation time lowered to
tau_out = 0.51 (tau_in = 0.6), so that Oh = mu_in / sqrt(rho sigma R0) is
about 0.07.  (At the benchmark's tau_out = 0.8, Oh is about 2.2: the
spreading is viscous and slower.)

The contact radius follows protocol (i) of Sec. III B: the mean distance from
its centre of the membrane's crossing of a plane parallel to the wall.  The
plane sits at the minimum of Pi(h), h* = xi (n/m)^(1/(n-m)) = 2^(1/3) xi,
where the paper finds the intersection height that best shows the inertial
law.  Time is measured in the inertial time t~ = sqrt(rho R0^3 / sigma).

After the onset (the paper sees it near t/t~ = 0.01) the radius grows as a
power law close to t^(1/2).  The test fits log r_c against log t over
t/t~ in [0.02, 0.4] and asks for an exponent within 0.1 of 1/2 (the
qualitative bar for a scaling law read off a log-log plot); r_c must grow
monotonically there and the run must stay stable."""
import math

import numpy as np
import pytest

from paper_2503_20605_gb300 import iblb
from paper_2503_20605_gb300 import inputs as I
from gpu_util import stream

pytestmark = pytest.mark.gpu

TAU_OUT, LAMBDA = 0.51, 10.0


@pytest.fixture(autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    iblb.lib()


def test_inertial_spreading_exponent():
    w = I.workload_spreading_256("bf16")
    lat = iblb.lattice_desc(w.nx, w.ny, w.nz, tau_out=TAU_OUT, lam=LAMBDA, storage="bf16")
    phys = iblb.physics_desc(sigma=w.sigma, theta_eq_deg=w.theta_deg, xi=w.xi, volume_correction=1)
    ctx = iblb.iblb_create(lat, phys, stream())
    t_tilde = math.sqrt(w.R ** 3 / w.sigma)
    zcut_frac = w.xi * 2.0 ** (1.0 / 3.0) / w.R
    every = 10
    ts, rc = [], []
    try:
        xyz, tri = w.mesh()
        iblb.iblb_set_membrane(ctx, 0, xyz, tri)
        done = 0
        while done < 0.4 * t_tilde:
            iblb.iblb_step(ctx, every)
            done += every
            o = iblb.iblb_observe(ctx, 0, zcut_frac, 0.1)
            assert o["status"] == 0, (done, o["status"])
            ts.append(done)
            rc.append(o["rc_cut"])
    finally:
        iblb.iblb_destroy(ctx)
    t = np.array(ts, np.float64) / t_tilde
    r = np.array(rc) / w.R
    for lo, hi in ((0.01, 0.05), (0.02, 0.1), (0.05, 0.2), (0.1, 0.4)):
        sel = (t >= lo) & (t <= hi)
        k = np.polyfit(np.log(t[sel]), np.log(r[sel]), 1)[0]
        print(f"t/t~ in [{lo}, {hi}]: exponent {k:.3f}, r_c/R0 {r[sel][0]:.3f} .. {r[sel][-1]:.3f}")
    sel = (t >= 0.02) & (t <= 0.4)
    assert np.all(r[sel] > 0) and np.all(np.diff(r[sel]) >= -1e-3), r[sel]
    k = np.polyfit(np.log(t[sel]), np.log(r[sel]), 1)[0]
    print(f"exponent over t/t~ in [0.02, 0.4]: {k:.3f}")
    assert abs(k - 0.5) <= 0.1, k
