"""Planted mistakes: the oracle's pins must be able to fail.

Each case copies the oracle (oracle/), the seeded input module and the pin
tests into a scratch directory, makes ONE plausible mistake in one oracle
file -- a dropped term, a wrong sign, factor or index, a transposed operand,
a shifted stencil -- and runs the pin files named beside it there.  The
pins must then report a failed assertion (not an import or build error:
each mutant is checked to compile before it runs).  Only pins against the
paper and the mathematics take part; the comparisons of the oracle with the
library's host code are deselected, since they would catch a mutant without
saying anything about the pins.

The mistakes cover every part of the oracle: the lattice equilibrium and
the Guo source (Sec. II A), the collision, streaming and bounce-back, the
kernel Psi and the spread / interpolation (eqs. force_spread,
vel_interpolation), the membrane's surface-tension and elastic forces
(Sec. II B), the wetting force and eq. A_choice (Sec. II C), the in/out ray
test, the mesh volume, area and eq. angleh, the time step's advection and
body force, the network's backward pass and Adam, the warm-start geometry,
and the App. B shape solver.  Each mutant is caught without the longer
physics runs (marked slow), which are left out to keep the set short; the
mutants run in parallel processes and the whole set takes about half a
minute."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

LAT, IB, MEM, INS, OBS, PHY = ("test_oracle_lattice.py", "test_oracle_ib.py", "test_oracle_membrane.py",
                               "test_oracle_inside.py", "test_oracle_observe.py", "test_oracle_physics.py")
MLP, SHP, WSG = "test_oracle_mlp.py", "test_oracle_shape.py", "test_warmstart_geometry.py"

# (name, file, anchor, old, new, pin files): the first `old` after `anchor`
# in `file` becomes `new`
MUTANTS = [
    ("feq_drops_quadratic_term", "oracle.c", "void orc_feq(",
     " + cu * cu / (2.0 * CS2 * CS2)", "", [LAT]),
    ("feq_sign_of_u_squared", "oracle.c", "void orc_feq(",
     "- uu / (2.0 * CS2)", "+ uu / (2.0 * CS2)", [LAT]),
    ("guo_drops_prefactor", "oracle.c", "void orc_guo_source(",
     "double pref = 1.0 - 1.0 / (2.0 * tau);", "double pref = 1.0;", [LAT]),
    ("guo_sign_of_u", "oracle.c", "void orc_guo_source(",
     "(C[i][a] - u[a]) / CS2", "(C[i][a] + u[a]) / CS2", [LAT]),
    ("guo_transposed_component", "oracle.c", "void orc_guo_source(",
     "cu / (CS2 * CS2) * C[i][a]", "cu / (CS2 * CS2) * C[i][(a + 1) % 3]", [LAT]),
    ("velocity_drops_half_force", "oracle.c", "void orc_collide_cell(",
     "(j[a] + 0.5 * F[a]) / rho", "j[a] / rho", [LAT]),
    ("collision_sign_of_source", "oracle.c", "void orc_collide_cell(",
     "/ tau + S[i];", "/ tau - S[i];", [LAT]),
    ("collision_relaxes_with_tau_squared", "oracle.c", "void orc_collide_cell(",
     "(f[i] - feq[i]) / tau", "(f[i] - feq[i]) / (tau * tau)", [LAT]),
    ("weights_swapped", "oracle.c", "static const double W[19]",
     "1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,",
     "1.0 / 36.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,", [LAT]),
    ("bounce_back_keeps_direction", "oracle.c", "static void one_step(",
     "f[i] = s->f[opposite(i) * cells + cell];", "f[i] = s->f[i * cells + cell];", [LAT]),
    ("streaming_pushes_instead_of_pulls", "oracle.c", "static void one_step(",
     "int sx = wrap1(x - C[i][0], nx)", "int sx = wrap1(x + C[i][0], nx)", [LAT]),
    ("body_force_dropped", "oracle.c", "static void one_step(",
     "s->F[a * cells + c] += p->body_force[a];", "(void)c;", [LAT]),
    ("psi_outer_branch_sign", "oracle.c", "double orc_psi(",
     "0.625 - 0.25 * r - 0.25 * sqrt(", "0.625 - 0.25 * r + 0.25 * sqrt(", [IB]),
    ("psi_inner_branch_constant", "oracle.c", "double orc_psi(",
     "0.375 - 0.25 * r", "0.375 - 0.125 * r", [IB]),
    ("spread_transposed_component", "oracle.c", "void orc_spread(",
     "phi[3 * j + a] * d", "phi[3 * j + (a + 1) % 3] * d", [IB]),
    ("spread_stencil_shifted", "oracle.c", "void orc_spread(",
     "X = b[0] - 1; X <= b[0] + 2", "X = b[0] - 2; X <= b[0] + 1", [IB]),
    ("interp_drops_z_weight", "oracle.c", "void orc_interp(",
     "double d = px * py * pz;", "double d = px * py;", [IB]),
    ("stencil_wall_layer_off_by_one", "oracle.c", "static int fluid_layer(",
     "(Z >= 1 && Z <= p->nz - 2) ? Z - 1 : -1", "(Z >= 0 && Z <= p->nz - 3) ? Z : -1", [IB]),
    ("tension_sign", "oracle.c", "int orc_membrane_forces(",
     "fs[a] = -p->sigma * gs[3 * j + a];", "fs[a] = p->sigma * gs[3 * j + a];", [MEM]),
    ("area_gradient_edge_reversed", "oracle.c", "int orc_membrane_forces(",
     "sub3(qprev, qnext, d);", "sub3(qnext, qprev, d);", [MEM]),
    ("wetting_share_half_not_third", "oracle.c", "int orc_membrane_forces(",
     "-(chi[j] / 3.0) * Pi", "-(chi[j] / 2.0) * Pi", [MEM]),
    ("wetting_wall_plane_at_one", "oracle.c", "int orc_membrane_forces(",
     "double h = xyz[3 * j + 2] - 0.5;", "double h = xyz[3 * j + 2] - 1.0;", [MEM]),
    ("A_choice_sign_of_cos", "oracle.c", "double orc_wetting_A(",
     "(1.0 + cos(theta))", "(1.0 - cos(theta))", [MEM]),
    ("Pi_exponents_swapped", "oracle.c", "double orc_Pi(",
     "pow(r, n) - pow(r, m)", "pow(r, m) - pow(r, n)", [MEM]),
    ("elastic_drops_area_modulus", "oracle.c", "void orc_membrane_elastic(",
     " + (ka / 3.0) * r * (r * r - 1.0)", "", [MEM]),
    ("elastic_sign_of_S12", "oracle.c", "void orc_membrane_elastic(",
     "S12 = -h12 / det", "S12 = h12 / det", [MEM]),
    ("elastic_shear_term_misses_2b", "oracle.c", "void orc_membrane_elastic(",
     "(2.0 * b + 1.0)", "(b + 1.0)", [MEM]),
    ("inside_sets_instead_of_toggling", "oracle.c", "void orc_inside(",
     "inside[cr[k].col + ncol * z] ^= 1;", "inside[cr[k].col + ncol * z] |= 1;", [INS]),
    ("inside_half_open_rule_closed", "oracle.c", "static int edge_keeps(",
     "return dy > 0.0 || (dy == 0.0 && dx < 0.0);", "return dy >= 0.0;", [INS]),
    ("inside_ignores_wall_layer", "oracle.c", "void orc_inside(",
     "double Z = p->walls ? z + 1 : z;", "double Z = z;", [INS]),
    ("volume_third_not_sixth", "oracle.c", "double orc_mesh_volume(",
     "return V / 6.0;", "return V / 3.0;", [OBS]),
    ("area_drops_half", "oracle.c", "double orc_mesh_area(",
     "A += 0.5 * sqrt(", "A += sqrt(", [OBS]),
    ("angleh_drops_factor_three", "oracle.c", "double orc_theta_from_height(",
     "sqrt(3.0 * l3 / (R3 - l3))", "sqrt(l3 / (R3 - l3))", [OBS]),
    ("contact_radius_uncentred", "oracle.c", "void orc_mesh_observe(",
     "sqrt((px - cx) * (px - cx) + (py - cy) * (py - cy))", "sqrt(px * px + py * py)", [OBS]),
    ("tau_inside_outside_swapped", "oracle.c", "static void one_step(",
     "in[c] ? p->tau_in : p->tau_out", "in[c] ? p->tau_out : p->tau_in", [PHY]),
    ("volume_correction_about_origin", "oracle.c", "static void one_step(",
     "s->q[3 * j + a] = c[a] + (s->q[3 * j + a] - c[a]) * k;", "s->q[3 * j + a] = s->q[3 * j + a] * k;", [OBS]),
    ("volume_correction_square_root", "oracle.c", "static void one_step(",
     "double k = cbrt(s->V0 / V);", "double k = sqrt(s->V0 / V);", [OBS]),
    ("advection_half_step", "oracle.c", "static void one_step(",
     "s->q[k] += s->qdot[k];", "s->q[k] += 0.5 * s->qdot[k];", [PHY]),
    ("mlp_tanh_derivative", "mlp.py", "def grad(",
     "(1.0 - acts[l] * acts[l])", "(1.0 - acts[l])", [MLP]),
    ("mlp_loss_scale", "mlp.py", "def grad(",
     "/ (S * n_out)", "/ S", [MLP]),
    ("mlp_bias_gradient_transposed", "mlp.py", "def grad(",
     "dz.sum(axis=0)", "dz.sum(axis=0)[::-1]", [MLP]),
    ("adam_no_bias_correction", "mlp.py", "def step(",
     "vh = self.v / (1.0 - BETA2 ** self.t)", "vh = self.v", [MLP]),
    ("mlp_feature_scale", "mlp.py", "def features(",
     "(x[:, 1] - 16.0) / 8.0", "(x[:, 1] - 16.0) / 6.0", [MLP]),
    ("cap_radius_sign", "warmstart.py", "def cap_profile(",
     "(2.0 - 3.0 * ct + ct ** 3)", "(2.0 - 3.0 * ct - ct ** 3)", [WSG]),
    ("cap_zone_height_third", "warmstart.py", "def cap_profile(",
     "z_s = 0.5 * hcap", "z_s = hcap / 3.0", [WSG]),
    ("deform_scale_not_cube_root", "warmstart.py", "def deform(",
     "s = np.cbrt(mesh_volume(d, tri) / mesh_volume(q, tri))",
     "s = np.sqrt(mesh_volume(d, tri) / mesh_volume(q, tri))", [WSG]),
    ("profile_bins_off_by_half", "warmstart.py", "def profile_at(",
     "(np.arange(nphi) + 0.5) * np.pi / nphi", "np.arange(nphi) * np.pi / nphi", [WSG]),
    ("curvature_factor_two", "shape.py", "def curvature(",
     "(u * gd + 3 * g)", "(u * gd + 2 * g)", [SHP]),
    ("wall_term_sign_of_cos", "shape.py", "def wall_term(",
     "(1.0 + np.cos(theta))", "(1.0 - np.cos(theta))", [SHP]),
    ("wall_term_prefactor", "shape.py", "def wall_term(",
     "(m - 1) * (n - 1) / ((n - m) * eps)", "(m - 1) * n / ((n - m) * eps)", [SHP]),
    ("curvature_second_term_dropped_u", "shape.py", "def curvature(",
     "(u * gd + 3 * g) / (g * Q)", "(3 * g) / (g * Q)", [SHP]),
    ("centroid_half_not_three_quarters", "shape.py", "def centroid_height(",
     "0.75 * np.trapezoid", "0.5 * np.trapezoid", [SHP]),
    ("shape_angleh_drops_factor_three", "shape.py", "def angle_from_height(",
     "np.sqrt(3.0 * ell ** 3", "np.sqrt(ell ** 3", [SHP]),
]

PINS_ONLY = "not library and not package"


def _scratch_tree(dst):
    """The oracle's sources, the seeded input module and the pin tests."""
    os.makedirs(os.path.join(dst, "oracle"))
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            shutil.copy2(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle", f))
    pkg = "paper_2503_20605_gb300"
    os.makedirs(os.path.join(dst, pkg))
    for f in ("__init__.py", "inputs.py"):
        shutil.copy2(os.path.join(ROOT, pkg, f), os.path.join(dst, pkg, f))
    os.makedirs(os.path.join(dst, "tests"))
    for f in os.listdir(os.path.join(ROOT, "tests")):
        pin_file = f.startswith("test_oracle_") and f != os.path.basename(__file__)
        if f in ("conftest.py", WSG) or pin_file:
            shutil.copy2(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))


def _plant(dst, fname, anchor, old, new):
    path = os.path.join(dst, "oracle", fname)
    with open(path) as f:
        src = f.read()
    a = src.index(anchor)
    k = src.index(old, a)
    src = src[:k] + new + src[k + len(old):]
    with open(path, "w") as f:
        f.write(src)
    if fname.endswith(".c"):
        subprocess.run(["gcc", "-std=c11", "-D_DEFAULT_SOURCE", "-fsyntax-only", path],
                       check=True, capture_output=True)
    else:
        compile(src, path, "exec")


def _run(base, m):
    name, fname, anchor, old, new, files = m
    dst = os.path.join(base, name)
    _scratch_tree(dst)
    _plant(dst, fname, anchor, old, new)
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    env["PYTHONDONTWRITEBYTECODE"] = "1"
    r = subprocess.run([sys.executable, "-m", "pytest", *[os.path.join("tests", f) for f in files], "-x", "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu and not slow", "-k", PINS_ONLY],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = str(tmp_path_factory.mktemp("mutants"))
    workers = max(2, min(8, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        futs = {m[0]: ex.submit(_run, base, m) for m in MUTANTS}
        return {k: f.result() for k, f in futs.items()}


def test_unmutated_pins_pass(tmp_path):
    """The scratch tree itself is sound: with no mistake planted, the pin
    files the mutants use all pass there."""
    _scratch_tree(str(tmp_path))
    files = sorted({f for m in MUTANTS for f in m[5]})
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    env["PYTHONDONTWRITEBYTECODE"] = "1"
    r = subprocess.run([sys.executable, "-m", "pytest", *[os.path.join("tests", f) for f in files], "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu and not slow", "-k", PINS_ONLY],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("m", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(outcomes, m):
    rc, out = outcomes[m[0]]
    tail = out.strip().splitlines()[-1] if out.strip() else ""
    # exit status 1: tests ran and at least one failed (2-5 are errors of
    # collection or usage, which would not show that a pin caught anything)
    # (an exception the mutant raises inside a pin's fixture, such as the
    # shape solver giving up, reports as an error of that pin and counts)
    assert rc == 1, (m[0], rc, out)
    assert "failed" in tail or " error" in tail, (m[0], tail)
