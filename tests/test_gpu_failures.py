"""Error paths of the C ABI on the GPU, made on the host side: invalid meshes
are refused before any device work, and conditions the kernels detect
(non-finite values, a node moving more than half a cell in one step, a node
leaving the fluid) come back from iblb_sync as IBLB_E_UNSTABLE with a
message, never as a device fault.  After each error the context is reset
through the API and runs on, bit for bit like a fresh context.  The bounded
wait of the stream-collide pipeline is made to run out on a barrier that
nothing completes: it reports IBLB_E_TIMEOUT and the device stays usable."""
import numpy as np
import pytest

from paper_2503_20605_gb300 import iblb
from paper_2503_20605_gb300 import inputs as I
from gpu_util import gpu_ctx

pytestmark = pytest.mark.gpu

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 0],
              [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1], [1, 0, 1],
              [-1, 0, -1], [1, 0, -1], [-1, 0, 1]], float)


@pytest.fixture(autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    iblb.lib()


def parity_ctx():
    w = I.workload_parity_32()
    xyz, tri = w.mesh()
    ctx = gpu_ctx(w.nx, w.ny, w.nz, tau=w.tau, sigma=w.sigma, theta=w.theta_deg, xi=w.xi, mesh=(xyz, tri))
    return ctx, xyz, tri


def rest(ctx):
    cells = iblb.iblb_info(ctx, 0)["cells"]
    return np.repeat(W, cells)


def test_invalid_meshes_are_refused():
    w = I.workload_parity_32()
    xyz, tri = w.mesh()
    ctx = gpu_ctx(w.nx, w.ny, w.nz, tau=w.tau, sigma=w.sigma, theta=w.theta_deg, xi=w.xi)
    try:
        bad = {"open": tri[1:], "inward": tri[:, ::-1].copy(), "index": np.where(tri == 5, len(xyz), tri)}
        for name, t in bad.items():
            with pytest.raises(iblb.IblbError) as e:
                iblb.iblb_set_membrane(ctx, 0, xyz, np.ascontiguousarray(t, np.int32))
            assert e.value.code in (iblb.IBLB_E_MESH, iblb.IBLB_E_ARG), name
        iblb.iblb_set_membrane(ctx, 0, xyz, tri)
        iblb.iblb_step(ctx, 5)
        iblb.iblb_sync(ctx)
    finally:
        iblb.iblb_destroy(ctx)


def run_clean(ctx, xyz, n):
    iblb.iblb_set_populations(ctx, 0, rest(ctx))
    iblb.iblb_set_nodes(ctx, 0, xyz)
    iblb.iblb_step(ctx, n)
    iblb.iblb_sync(ctx)
    return iblb.iblb_get_nodes(ctx, 0), iblb.iblb_get_populations(ctx, 0)


def expect_unstable(ctx, words):
    with pytest.raises(iblb.IblbError) as e:
        iblb.iblb_sync(ctx)
    assert e.value.code == iblb.IBLB_E_UNSTABLE
    assert words in str(e.value)


def test_device_conditions_report_and_recover():
    ctx, xyz, tri = parity_ctx()
    fresh, _, _ = parity_ctx()
    try:
        q_ref, f_ref = run_clean(fresh, xyz, 20)
        nx, ny = 32, 32
        cells = iblb.iblb_info(ctx, 0)["cells"]

        # a non-finite population next to the lowest node
        f = rest(ctx)
        j = int(np.argmin(xyz[:, 2]))
        x, y, zf = int(xyz[j, 0]), int(xyz[j, 1]), int(xyz[j, 2]) - 1
        f[np.arange(19) * cells + x + nx * (y + ny * zf)] = np.nan
        iblb.iblb_set_populations(ctx, 0, f)
        iblb.iblb_step(ctx, 3)
        expect_unstable(ctx, "non-finite")
        q, fpop = run_clean(ctx, xyz, 20)
        np.testing.assert_array_equal(q, q_ref)
        np.testing.assert_array_equal(fpop, f_ref)

        # a uniform flow of 0.6 per step in x moves every node too far
        u = np.array([0.6, 0.0, 0.0])
        cu = C @ u
        feq = W * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u @ u)
        iblb.iblb_set_populations(ctx, 0, np.repeat(feq, cells))
        iblb.iblb_step(ctx, 1)
        expect_unstable(ctx, "more than 1/2")
        q, fpop = run_clean(ctx, xyz, 20)
        np.testing.assert_array_equal(q, q_ref)

        # a node placed far above the box leaves the fluid
        moved = xyz.copy()
        moved[0, 2] = 500.0
        iblb.iblb_set_populations(ctx, 0, rest(ctx))
        iblb.iblb_set_nodes(ctx, 0, moved)
        iblb.iblb_step(ctx, 1)
        expect_unstable(ctx, "left the fluid")
        q, fpop = run_clean(ctx, xyz, 20)
        np.testing.assert_array_equal(q, q_ref)
        np.testing.assert_array_equal(fpop, f_ref)
    finally:
        iblb.iblb_destroy(ctx)
        iblb.iblb_destroy(fresh)


def test_bounded_wait_runs_out_and_reports():
    from gpu_util import stream
    # about 1 ms at GB300 clocks: the wait gives up, every thread reports it
    assert iblb.iblb_selftest_wait_timeout(2_000_000, stream()) == iblb.IBLB_E_TIMEOUT
    assert iblb.iblb_selftest_wait_timeout(10, stream()) == iblb.IBLB_E_ARG
    # the context is still usable: a clean run matches a fresh one bit for bit
    ctx, xyz, tri = parity_ctx()
    fresh, _, _ = parity_ctx()
    try:
        q_ref, f_ref = run_clean(fresh, xyz, 5)
        q, f = run_clean(ctx, xyz, 5)
        np.testing.assert_array_equal(q, q_ref)
        np.testing.assert_array_equal(f, f_ref)
    finally:
        iblb.iblb_destroy(ctx)
        iblb.iblb_destroy(fresh)

