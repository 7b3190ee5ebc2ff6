"""Simulated equilibrium shapes against the axisymmetric theory (Sec. III A,
App. B), through the C ABI.

The paper's statics setting: an 80 x 80 x 60 box (periodic in x and y,
bounce-back walls), lambda = 1, R0 = 20, theta_eq in {pi/4, pi/2, 3pi/4},
xi/R0 in {0.2, 0.3}, a sphere started just above the wall.  The mesh is the
level-5 icosphere (20 480 triangles, the paper's coarser N_t = 20 000); the
six droplets run as one batched context until the contact angle (eq.
angleh) changes by less than 0.05 degree over 2000 steps.  Then:

* G_sim(phi): the distance of every node from the droplet's volume centroid,
  averaged over the azimuth in 48 bins of the polar angle phi;
* G_theo(phi): the solution of eq. YL for the same theta_eq and xi/R0
  (oracle/shape.py, R0 the radius of the sphere of the simulated volume),
  measured from its own volume centroid in the same way;
* eq. L2-error_equilibrium between the two must stay at or below 0.01, the
  largest error the paper reports for a well-resolved interface (its error
  figure for the statics); the contact angles of both (eq. angleh) must
  agree within 1.5 degrees; at theta_eq = pi/4 the error must grow as xi/R0
  decreases, the paper's trend.

Both storages are run: FP32 and FP16 offsets (the reduced-precision path
must reach the same shape).  Two more runs: the error must fall with the
membrane's resolution (the paper's study of N_t), and the 128^3 benchmark
droplet (xi/R0 = 0.1) must reach the theory's shapes and angles at five
contact angles, its error falling as theta_eq grows."""
import math

import numpy as np
import pytest

import oracle.shape as S
from paper_2503_20605_gb300 import iblb
from paper_2503_20605_gb300 import inputs as I
from gpu_util import stream

pytestmark = pytest.mark.gpu

CASES = [(t, e) for t in (45.0, 90.0, 135.0) for e in (0.2, 0.3)]
R0, SIGMA, NBIN = 20.0, 0.01, 48
E_L2_BAR, ANGLE_BAR_DEG = 0.01, 1.5


@pytest.fixture(autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    iblb.lib()


def volume_centroid(xyz, tri):
    """Centroid of the closed surface's enclosed volume (sum over the
    tetrahedra from the origin to each outward-oriented triangle)."""
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    v = np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0
    return (v[:, None] * (a + b + c) / 4.0).sum(0) / v.sum(), v.sum()


def sim_profile(xyz, tri, edges):
    """Azimuthally averaged node distance from the centroid per phi bin (a
    bin without nodes, which a flat droplet can leave near its poles, takes
    the linear interpolation of its filled neighbours)."""
    c, vol = volume_centroid(xyz, tri)
    d = xyz - c
    r = np.linalg.norm(d, axis=1)
    phi = np.arccos(np.clip(d[:, 2] / r, -1.0, 1.0))
    idx = np.clip(np.digitize(phi, edges) - 1, 0, len(edges) - 2)
    cnt = np.bincount(idx, minlength=len(edges) - 1)
    assert (cnt > 0).sum() >= 0.9 * len(cnt), cnt
    g = np.bincount(idx, weights=r, minlength=len(edges) - 1) / np.maximum(cnt, 1)
    mids = 0.5 * (edges[1:] + edges[:-1])
    full = cnt > 0
    return np.interp(mids, mids[full], g[full]), vol


def run_statics(specs, storage):
    """Run the droplets as one batched context until each one's contact
    angle moved less than 0.05 degree over 2000 steps; returns per droplet
    (equilibrium step, nodes, triangles, angle)."""
    lats = [iblb.lattice_desc(s.nx, s.ny, s.nz, tau_out=s.tau, storage=storage) for s in specs]
    phys = [iblb.physics_desc(sigma=s.sigma, theta_eq_deg=s.theta_deg, xi=s.xi, volume_correction=1)
            for s in specs]
    ctx = iblb.iblb_batch_create(lats, phys, stream())
    n = len(specs)
    tris = []
    hist = [[] for _ in range(n)]
    eq = np.full(n, -1)
    nodes = [None] * n
    theta_sim = np.full(n, np.nan)
    try:
        for k, s in enumerate(specs):
            xyz, tri = s.mesh()
            tris.append(tri)
            iblb.iblb_set_membrane(ctx, k, xyz, tri)
        done, every, lag = 0, 500, 4
        while done < 60000 and np.any(eq < 0):
            iblb.iblb_step(ctx, every)
            done += every
            for k, o in enumerate(iblb.iblb_observe_all(ctx)):
                assert o["status"] == 0, (storage, k, done, o["status"])
                if eq[k] >= 0:
                    continue
                hist[k].append(o["theta_RV_deg"])
                if done >= 4000 and abs(hist[k][-1] - hist[k][-1 - lag]) < 0.05:
                    eq[k] = done
                    nodes[k] = iblb.iblb_get_nodes(ctx, k)
                    theta_sim[k] = o["theta_RV_deg"]
    finally:
        iblb.iblb_destroy(ctx)
    assert np.all(eq > 0), eq
    return eq, nodes, tris, theta_sim


def shape_error(nodes, tri, theta_deg, xi, nbin=NBIN):
    """Eq. L2-error_equilibrium of one equilibrium against the theory, and
    the theory's angle."""
    edges = np.linspace(0.0, np.pi, nbin + 1)
    mids = 0.5 * (edges[1:] + edges[:-1])
    g_sim, vol = sim_profile(nodes, tri, edges)
    r0 = (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)
    u, g, _, _ = S.solve(math.radians(theta_deg), xi / r0, n_grid=801)
    return S.e_l2(mids, g_sim / r0, S.profile_about_centroid(u, g, mids)), math.degrees(S.angle_from_height(g))


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_equilibrium_shape_matches_theory(storage):
    specs = [I.DropletSpec(80, 80, 60, R0, 5, SIGMA, t, e * R0, tau=1.0, storage=storage) for t, e in CASES]
    eq, nodes, tris, theta_sim = run_statics(specs, storage)
    rows = []
    for k, (t, e) in enumerate(CASES):
        err, th_theo = shape_error(nodes[k], tris[k], t, specs[k].xi)
        rows.append((t, e, eq[k], err, theta_sim[k], th_theo))
    print(storage, "theta_eq, xi/R0, steps, E_L2, theta_sim, theta_theory:")
    for r in rows:
        print("  %5.1f %.1f %6d %.5f %7.3f %7.3f" % r)
    for t, e, _, err, ths, tht in rows:
        assert err <= E_L2_BAR, (storage, t, e, err)
        assert abs(ths - tht) <= ANGLE_BAR_DEG, (storage, t, e, ths, tht)
    # the paper's trend for the smallest angle: the error grows as xi/R0
    # decreases (its error figure; at 3 pi/4 it does not depend on xi/R0)
    err = {(row[0], row[1]): row[3] for row in rows}
    assert err[(45.0, 0.2)] > err[(45.0, 0.3)], err


def test_error_falls_with_mesh_resolution():
    # the paper's resolution study: a finer membrane gives a smaller error;
    # theta_eq = pi/4, xi/R0 = 0.2 with 5 120 and 20 480 triangles (a finer
    # level would put more nodes over a 4^3 tile than its list holds); both
    # profiles in 24 bins of phi, so that the coarse mesh fills every bin
    specs = [I.DropletSpec(80, 80, 60, R0, lvl, SIGMA, 45.0, 0.2 * R0, tau=1.0, storage="f32") for lvl in (4, 5)]
    eq, nodes, tris, theta_sim = run_statics(specs, "f32")
    errs = [shape_error(nodes[k], tris[k], 45.0, specs[k].xi, nbin=24)[0] for k in range(2)]
    print("E_L2 with 5 120 and 20 480 triangles:", errs, "steps", eq, "angles", theta_sim)
    assert errs[1] < errs[0], errs


def test_benchmark_droplet_reaches_theory():
    # the 128^3 benchmark droplet (R0 = 24, xi/R0 = 0.1, 20 480 triangles,
    # FP16 storage) at theta_eq = 30 .. 150 degrees, with sigma = 0.01 to
    # settle sooner: the shape error falls as theta_eq grows (the paper's
    # trend at a small xi/R0), within 0.01 from 60 degrees on and 0.02 at 30,
    # and the angles agree with the theory's within 2 degrees
    angles = [30.0, 60.0, 90.0, 120.0, 150.0]
    specs = [I.workload_statics_128(t, "f16") for t in angles]
    for s in specs:
        s.sigma = SIGMA
    eq, nodes, tris, theta_sim = run_statics(specs, "f16")
    rows = [(t,) + shape_error(nodes[k], tris[k], t, specs[k].xi) for k, t in enumerate(angles)]
    for (t, err, tht), ths, n in zip(rows, theta_sim, eq):
        print(f"theta_eq {t:5.1f}: {n} steps, E_L2 {err:.5f}, theta {ths:.3f} (theory {tht:.3f})")
    errs = [r[1] for r in rows]
    assert errs[0] <= 0.02 and max(errs[1:]) <= E_L2_BAR, errs
    assert all(errs[k + 1] < errs[k] for k in range(len(errs) - 1)), errs
    assert max(abs(ths - r[2]) for r, ths in zip(rows, theta_sim)) <= 2.0, (rows, theta_sim)
