"""Late-stage spreading from a spherical-cap start (Sec. III B, Fig. 5b)
through the C ABI.

The paper bypasses the inertial stage by starting from a spherical cap and
sees the contact radius approach Tanner's law r_c ~ t^(1/10) (viscous
spreading) before the droplet settles; the separation of the regularising
length xi from R0 matters (xi = 3 there).  The run here: R0 = 60, xi = 3, an
L7 icosphere (163 842 nodes, 327 680 faces: the paper's mesh densities)
deformed to the hemispherical cap, theta_eq = pi/8, tau = 1 (lambda = 1),
sigma = 0.01, volume correction on, FP16 offsets, in a 320 x 320 x 98 box
(paper_2503_20605_gb300.tanner).  Time in t* = mu R0 / sigma = 1000 steps,
contact radius by protocol (i) at h* = 2^(1/3) xi.

A 150 000-step run of the same set-up measured a fitted exponent of 0.096
over t/t* in [3, 10], 0.11 over [5, 30] and 0.107 over [10, 30], then a
slow-down as the angle nears its equilibrium (0.04 over [30, 100]).  The
test runs 30 000 steps and asks for an exponent within 0.03 of 1/10 over
t/t* in [5, 30], a monotonically growing radius, an unchanged volume and no
device status (no tile-list or column overflow at these mesh densities)."""
import numpy as np
import pytest

from paper_2503_20605_gb300 import iblb
from paper_2503_20605_gb300 import tanner as T
from gpu_util import stream

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    iblb.lib()


def test_tanner_exponent_from_cap_start():
    res = T.run(R0=60.0, theta_eq_deg=22.5, theta0_deg=90.0, xi=3.0, level=7, steps=30000, every=500,
                storage="f16", stream=stream())
    assert res["status"] == 0, res["status"]
    t, r = np.array(res["t"]), np.array(res["rc"])
    assert np.all(np.diff(r) > 0), r
    assert np.abs(np.array(res["volume_ratio"]) - 1.0).max() < 1e-9
    sel = (t >= 5.0) & (t <= 30.0)
    k = np.polyfit(np.log(t[sel]), np.log(r[sel]), 1)[0]
    print(f"Tanner window t/t* in [5, 30]: exponent {k:.3f}, r_c/R0 {r[sel][0]:.3f} .. {r[sel][-1]:.3f}, "
          f"{res['seconds']:.1f} s")
    assert abs(k - 0.1) <= 0.03, k
