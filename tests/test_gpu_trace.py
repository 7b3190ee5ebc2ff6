"""Per-warp tracing of one step (iblb_trace_step) through the C ABI: the
kernels start in the step's order, a kernel's end is the next one's first
start, and a traced step changes no result bit."""
import numpy as np
import pytest

from paper_2503_20605_gb300 import iblb
from paper_2503_20605_gb300 import inputs as I
from gpu_util import stream

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    iblb.lib()


def _ctx(volcorr):
    s = I.DropletSpec(40, 36, 30, 8.0, 3, 0.01, 70.0, 2.0, tau=0.9)
    lat = iblb.lattice_desc(s.nx, s.ny, s.nz, tau_out=s.tau, storage="f16")
    phys = iblb.physics_desc(sigma=s.sigma, theta_eq_deg=s.theta_deg, xi=s.xi, volume_correction=volcorr)
    c = iblb.iblb_create(lat, phys, stream())
    iblb.iblb_set_membrane(c, 0, *s.mesh())
    return c


def test_trace_orders_the_kernels_and_changes_nothing():
    plain, traced = _ctx(1), _ctx(1)
    try:
        iblb.iblb_step(plain, 12)
        iblb.iblb_step(traced, 5)
        trs = [iblb.iblb_trace_step(traced) for _ in range(3)]
        iblb.iblb_step(traced, 4)
        for c in (plain, traced):
            iblb.iblb_sync(c)
        assert np.array_equal(iblb.iblb_get_populations(plain, 0), iblb.iblb_get_populations(traced, 0))
        assert np.array_equal(iblb.iblb_get_nodes(plain, 0), iblb.iblb_get_nodes(traced, 0))
    finally:
        iblb.iblb_destroy(plain)
        iblb.iblb_destroy(traced)
    for tr in trs:
        names = iblb.TRACE_KERNELS
        assert all(tr[k] is not None and tr[k]["warps"] > 0 for k in names), tr
        assert tr["force"]["first_start_us"] == 0.0
        for k in names:
            t = tr[k]
            assert t["first_start_us"] <= t["median_start_us"] <= t["last_start_us"] <= t["end_us"], (k, tr)
        for prev, nxt in zip(names, names[1:]):
            assert tr[prev]["end_us"] == tr[nxt]["first_start_us"]
        print({k: round(tr[k]["end_us"] - tr[k]["first_start_us"], 2) for k in names})


def test_trace_without_volume_correction_reports_no_correction_kernel():
    c = _ctx(0)
    try:
        iblb.iblb_step(c, 2)
        tr = iblb.iblb_trace_step(c)
    finally:
        iblb.iblb_destroy(c)
    assert tr["vc"] is None
    assert tr["lb"]["end_us"] == tr["interp"]["first_start_us"]
    assert tr["interp"]["end_us"] >= tr["interp"]["last_start_us"]
