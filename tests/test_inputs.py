"""The seeded input generators hold the recipe the tests and the benchmark
use: icosphere sizes and geometry, the workloads' boxes and parameters, the
batch and warm-start distributions, and their determinism by seed."""
import math

import numpy as np
import pytest

from paper_2503_20605_gb300 import inputs as I


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_icosphere_counts_and_geometry(level):
    xyz, tri = I.icosphere(level, 7.0, (1.0, 2.0, 3.0))
    assert len(xyz) == 10 * 4 ** level + 2 and len(tri) == 20 * 4 ** level
    r = np.linalg.norm(xyz - [1.0, 2.0, 3.0], axis=1)
    assert np.allclose(r, 7.0, rtol=1e-14)
    # closed and consistently oriented: every directed edge once, its
    # reverse once; Euler characteristic V - E + F = 2
    edges = {(int(t[k]), int(t[(k + 1) % 3])) for t in tri for k in range(3)}
    assert len(edges) == 3 * len(tri)
    assert all((b, a) in edges for a, b in edges)
    assert len(xyz) - len(edges) // 2 + len(tri) == 2
    # faces counter-clockwise seen from outside: positive volume, below the sphere's
    a, b, c = xyz[tri[:, 0]] - [1, 2, 3], xyz[tri[:, 1]] - [1, 2, 3], xyz[tri[:, 2]] - [1, 2, 3]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    assert 0 < vol < 4.0 / 3.0 * math.pi * 343.0


def test_level_for_radius_keeps_edges_near_one_cell():
    # mean edge of an icosphere of level L and radius R is about 1.2 R / 2^L
    for R in np.linspace(6.0, 24.0, 37):
        L = I.level_for_radius(R)
        xyz, tri = I.icosphere(L, R)
        e = np.linalg.norm(xyz[tri[:, 0]] - xyz[tri[:, 1]], axis=1).mean()
        assert 0.5 < e < 1.5, (R, L, e)


def test_workloads_match_their_descriptions():
    w = I.workload_parity_32()
    assert (w.nx, w.ny, w.nz, w.R, w.level, w.theta_deg, w.xi) == (32, 32, 32, 8.0, 3, 90.0, 2.0)
    w = I.workload_statics_128(60.0)
    assert (w.nx, w.ny, w.nz, w.R, w.level, w.xi, w.storage) == (128, 128, 128, 24.0, 5, 2.4, "f16")
    w = I.workload_spreading_256()
    assert (w.nx, w.ny, w.nz, w.R, w.level, w.theta_deg, w.lam) == (256, 256, 128, 40.0, 6, 20.0, 10.0)
    assert math.isclose(w.tau_in, 0.5 + 10.0 * 0.3)
    # the droplet starts with its lowest node at h = xi above the wall plane
    for w in (I.workload_parity_32(), I.workload_statics_128(), I.workload_spreading_256()):
        xyz, _ = w.mesh()
        assert math.isclose(xyz[:, 2].min() - 0.5, w.xi, rel_tol=1e-12)
        assert math.isclose(xyz[:, 0].mean(), w.nx / 2.0, abs_tol=1e-9)


def test_batch_distribution_and_seed():
    b = I.workload_batch()
    assert len(b) == 64
    s = np.array([d.nx for d in b])
    assert s.min() >= 48 and s.max() <= 96 and all(d.nx == d.ny == d.nz for d in b)
    assert all(6.0 <= d.R <= 20.0 and 20.0 <= d.theta_deg <= 160.0 and 0.6 <= d.tau <= 1.2 for d in b)
    assert all(d.xi == max(2.0, 0.1 * d.R) and d.level == I.level_for_radius(d.R) for d in b)
    # every droplet fits its box with the wall gap and a margin
    assert all(2 * d.R + d.xi + 2 < d.nz for d in b)
    again = I.workload_batch()
    assert [(d.nx, d.R, d.theta_deg, d.tau) for d in b] == [(d.nx, d.R, d.theta_deg, d.tau) for d in again]
    other = I.workload_batch(seed=7)
    assert [d.R for d in other] != [d.R for d in b]


def test_warmstart_cases_and_perturbations():
    x = I.warmstart_cases(2000, 1)
    assert x.shape == (2000, 3)
    assert x[:, 0].min() >= 20 and x[:, 0].max() <= 160
    assert x[:, 1].min() >= 8 and x[:, 1].max() <= 24
    assert x[:, 2].min() >= 0.1 and x[:, 2].max() <= 10
    # log-uniform viscosity ratio: about half the cases below 1
    assert abs(np.mean(x[:, 2] < 1.0) - 0.5) < 0.05
    assert np.array_equal(x, I.warmstart_cases(2000, 1))
    w = np.full(19, 1.0 / 19.0)
    f = I.perturbed_populations(50, w, seed=3, amp=1e-2).reshape(19, 50)
    assert np.all(np.abs(f / w[:, None] - 1.0) <= 1e-2)
    assert np.array_equal(f.ravel(), I.perturbed_populations(50, w, seed=3, amp=1e-2))
    p = I.mlp_init(0)
    assert p.dtype == np.float32 and p.size == sum(o * i + o for i, o in zip(I.MLP_SIZES[:-1], I.MLP_SIZES[1:]))
    assert np.all(p[-64:] == 1.0)          # output biases: the sphere, g = 1
