"""The allocation-free mesh observables call (iblb_mesh_observe_dev_noalloc)
against the allocating one (iblb_mesh_observe_dev) through the C ABI: same
kernels, same launch shapes, so the results must agree to the last bits;
the test allows 1e-12 relative.  Two calls in a row on the same mesh, a
second mesh of another size in between, and the size limit.  Kept in a file
of its own, collected last, so that it also runs after every other GPU test
has used the device."""
import numpy as np
import pytest

from paper_2503_20605_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_20605_gb300 import build
    build.build()
    from paper_2503_20605_gb300 import iblb
    iblb.lib()
    return torch, iblb


def _mesh(torch, level, R, seed):
    xyz, tri = I.icosphere(level, R, (20.0, 21.0, 0.8 * R))
    xyz = I.jitter_nodes(xyz, seed, 0.05)
    d_xyz = torch.tensor(xyz, dtype=torch.float64, device="cuda").contiguous()
    d_tri = torch.tensor(tri, dtype=torch.int32, device="cuda").contiguous()
    return d_xyz, d_tri, len(xyz), len(tri)


def _both(torch, iblb, m, R0):
    d_xyz, d_tri, n, nt = m
    s = torch.cuda.current_stream().cuda_stream
    ref = iblb.iblb_mesh_observe_dev(d_xyz.data_ptr(), n, d_tri.data_ptr(), nt, R0, 0.05, 0.1, s)
    a = iblb.iblb_mesh_observe_dev_noalloc(d_xyz.data_ptr(), n, d_tri.data_ptr(), nt, R0, 0.05, 0.1, s)
    b = iblb.iblb_mesh_observe_dev_noalloc(d_xyz.data_ptr(), n, d_tri.data_ptr(), nt, R0, 0.05, 0.1, s)
    return ref, a, b


def test_noalloc_matches_allocating_call(env):
    torch, iblb = env
    big = _mesh(torch, 5, 24.0, 3)      # 20480 faces: 10 reduction chunks
    small = _mesh(torch, 2, 6.0, 4)     # 320 faces: one chunk
    for m, R0 in ((big, 24.0), (small, 6.0), (big, 24.0)):
        ref, a, b = _both(torch, iblb, m, R0)
        assert np.all(np.isfinite(ref))
        assert ref[0] > 0 and ref[1] > 0 and ref[11] > 0   # volume, area, crossing count
        np.testing.assert_allclose(a, ref, rtol=RTOL, atol=RTOL * np.abs(ref).max())
        np.testing.assert_allclose(b, ref, rtol=RTOL, atol=RTOL * np.abs(ref).max())


def test_noalloc_rejects_meshes_beyond_its_scratch(env):
    torch, iblb = env
    d_xyz, d_tri, n, nt = _mesh(torch, 1, 4.0, 5)
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(iblb.IblbError) as e:
        iblb.iblb_mesh_observe_dev_noalloc(d_xyz.data_ptr(), n, d_tri.data_ptr(), 1048577, 4.0, 0.05, 0.1, s)
    assert e.value.code == iblb.IBLB_E_ARG
    assert "static scratch" in str(e.value)
    with pytest.raises(iblb.IblbError) as e:
        iblb.iblb_mesh_observe_dev_noalloc(d_xyz.data_ptr(), 524289, d_tri.data_ptr(), nt, 4.0, 0.05, 0.1, s)
    assert e.value.code == iblb.IBLB_E_ARG
    # the call still works after a rejected one
    ref, a, _ = _both(torch, iblb, (d_xyz, d_tri, n, nt), 4.0)
    np.testing.assert_allclose(a, ref, rtol=RTOL, atol=RTOL * np.abs(ref).max())


def test_noalloc_with_device_memory_exhausted(env):
    """The use the call exists for: a caching allocator (torch's, here) holds
    every free byte of device memory, so that any further allocation fails.
    After one earlier call in this context (which did the set-up), the call
    still works and gives the same bits as before memory ran out."""
    torch, iblb = env
    m = _mesh(torch, 4, 12.0, 6)
    d_xyz, d_tri, n, nt = m
    ref, a, _ = _both(torch, iblb, m, 12.0)        # the warm-up call is among these
    s = torch.cuda.current_stream().cuda_stream
    hog, got = [], []
    try:
        chunk = 1 << 32
        while chunk >= 1 << 20:
            try:
                hog.append(torch.empty(chunk, dtype=torch.uint8, device="cuda"))
            except torch.cuda.OutOfMemoryError:
                chunk //= 2
        with pytest.raises(torch.cuda.OutOfMemoryError):
            torch.empty(2 << 20, dtype=torch.uint8, device="cuda")
        for _ in range(2):
            got.append(iblb.iblb_mesh_observe_dev_noalloc(d_xyz.data_ptr(), n, d_tri.data_ptr(), nt, 12.0,
                                                          0.05, 0.1, s))
    finally:
        del hog
        torch.cuda.empty_cache()
    for g in got:
        np.testing.assert_allclose(g, ref, rtol=RTOL, atol=RTOL * np.abs(ref).max())
