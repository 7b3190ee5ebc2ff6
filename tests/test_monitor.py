"""The diagnostics log's host logic on the CPU, with the library's step and
observables replaced by a fake: chunking of the steps, one JSON line per
droplet and interval, the volume ratio against the first observation, the
half-height, and the stop on a droplet error."""
import json

import pytest

from paper_2503_20605_gb300 import iblb, monitor


class FakeCtx:
    def __init__(self, fail_at=None):
        self.t, self.calls, self.fail_at = 0, [], fail_at

    def step(self, ctx, n):
        assert ctx is self
        self.calls.append(n)
        self.t += n

    def observe_all(self, ctx):
        out = []
        for k in range(2):
            st = iblb.IBLB_E_UNSTABLE if self.fail_at is not None and self.t >= self.fail_at and k == 1 else 0
            out.append({"mass": 100.0, "volume": 50.0 - 0.01 * self.t - k, "area": 60.0, "zmin": 2.5,
                        "zmax": 20.5 - 0.1 * k, "theta_R0_deg": 90.0, "theta_RV_deg": 91.0, "rc_cut": 5.0,
                        "rc_flat": 4.0, "n_cut": 30.0, "chi_flat": 12.0, "clamped": 0, "status": st})
        return out


def test_chunks_lines_and_ratios(tmp_path):
    f = FakeCtx()
    path = tmp_path / "log.jsonl"
    recs = monitor.run_logged(f, 25, 10, str(path), step=f.step, observe_all=f.observe_all)
    assert f.calls == [10, 10, 5]
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert lines == recs and len(lines) == 8
    assert [r["step"] for r in lines] == [0, 0, 10, 10, 20, 20, 25, 25]
    assert [r["droplet"] for r in lines] == [0, 1] * 4
    last = lines[-1]
    assert last["volume_ratio"] == pytest.approx((49.0 - 0.25) / 49.0)
    assert last["ell"] == pytest.approx(0.5 * (20.4 - 2.5))
    # appended, not overwritten
    monitor.run_logged(f, 0, 10, str(path), step=f.step, observe_all=f.observe_all)
    assert len(path.read_text().splitlines()) == 10


def test_stops_on_droplet_error(tmp_path):
    f = FakeCtx(fail_at=20)
    recs = monitor.run_logged(f, 100, 10, str(tmp_path / "e.jsonl"), step=f.step, observe_all=f.observe_all)
    assert f.calls == [10, 10]
    assert recs[-1]["step"] == 20 and recs[-1]["status"] == iblb.IBLB_E_UNSTABLE
    f2 = FakeCtx(fail_at=20)
    monitor.run_logged(f2, 40, 10, str(tmp_path / "k.jsonl"), stop_on_error=False, step=f2.step,
                       observe_all=f2.observe_all)
    assert f2.calls == [10, 10, 10, 10]


def test_rejects_bad_intervals(tmp_path):
    with pytest.raises(ValueError):
        monitor.run_logged(None, 10, 0, str(tmp_path / "x.jsonl"))


def test_fields_exist_in_the_library_observation():
    # the observation dict the binding builds from the C struct (no GPU
    # needed to build it) carries every field the log writes
    d = iblb.Obs().as_dict()
    assert set(monitor.FIELDS) <= set(d)
    r = monitor.record(0, 0, d, 0.0)
    assert r["volume_ratio"] is None and r["ell"] == 0.0


@pytest.mark.gpu
def test_log_of_a_real_context(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_20605_gb300 import inputs as I
    w = I.workload_parity_32()
    ctx = iblb.iblb_create(iblb.lattice_desc(w.nx, w.ny, w.nz, tau_out=w.tau),
                           iblb.physics_desc(sigma=w.sigma, theta_eq_deg=w.theta_deg, xi=w.xi),
                           torch.cuda.current_stream().cuda_stream)
    try:
        iblb.iblb_set_membrane(ctx, 0, *w.mesh())
        recs = monitor.run_logged(ctx, 20, 10, str(tmp_path / "p.jsonl"))
    finally:
        iblb.iblb_destroy(ctx)
    assert [r["step"] for r in recs] == [0, 10, 20]
    assert all(r["status"] == 0 for r in recs)
    assert abs(recs[-1]["volume_ratio"] - 1.0) < 1e-2 and recs[-1]["theta_RV_deg"] < 180.0 + 1e-9
