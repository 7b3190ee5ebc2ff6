"""Throughput of the IB-LB wetting time step on GB300.

Workload (default): the 128^3 statics droplet -- D3Q19, tau = 1, walls at
Z = 0 and Z = 127, L5 icosphere (10 242 nodes, 20 480 faces), R = 24,
sigma = 0.005, xi = 2.4, theta_eq = 90 deg, volume correction on -- with
populations stored as FP16 offsets (the headline) and, as a second line of
numbers in the same JSON, as FP32.  One step = the whole hot path: nodal
forces, binned spread, stream-collide, interpolation + advection, FP64 mesh
reductions + volume correction.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Value: MLUPS = fluid cells x steps / device time of the steps (CUDA events on
the library's stream), L2 flushed between timed steps.  Under torchrun each
rank runs its own replica of the workload (the droplet does not shard; the
value sums the cells of all ranks over the slowest rank's time).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and IB nodes/s at 128^3; FP16-store vs FP32 at <=1 deg contact-angle error"
BYTES_PER_CELL = {"f32": 152, "f16": 76, "bf16": 76}
FLUSH_BYTES = 512 << 20          # > 129 MB L2


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x, world, device):
    """Largest value of x over the ranks of the process group (x itself
    for one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells_per_rank, steps, max_step_ms, world):
    """Cells updated by all ranks (one replica each) over the slowest
    rank's time."""
    return world * cells_per_rank * steps / (max_step_ms * 1e-3) / 1e6


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def lb_source_sha():
    h = hashlib.sha1()
    for f in ("lb.cu", "iblb_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2503_20605_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def ncu_traffic(storage):
    """DRAM bytes per launch of the stream-collide kernel from the committed
    ncu capture (profiles/traffic.json), if it was taken on the current
    kernel source; None otherwise."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get("lb_kernel", {}).get(storage)
    if not e or e.get("source_sha") != lb_source_sha():
        return None
    return float(e["traffic_bytes_per_launch"])


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out = ""

    def summary(self):
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_ctx(iblb, spec, storage, stream):
    """One context for a droplet spec, or a batched context for a list."""
    specs = spec if isinstance(spec, list) else [spec]
    lats = [iblb.lattice_desc(w.nx, w.ny, w.nz, tau_out=w.tau, lam=w.lam, storage=storage) for w in specs]
    phys = [iblb.physics_desc(sigma=w.sigma, theta_eq_deg=w.theta_deg, xi=w.xi,
                              volume_correction=int(w.volume_correction)) for w in specs]
    if len(specs) == 1:
        ctx = iblb.iblb_create(lats[0], phys[0], stream)
    else:
        ctx = iblb.iblb_batch_create(lats, phys, stream)
    for k, w in enumerate(specs):
        xyz, tri = w.mesh()
        iblb.iblb_set_membrane(ctx, k, xyz, tri)
    xyz, tri = specs[0].mesh()
    return ctx, xyz, tri


def launches_per_step(spec):
    specs = spec if isinstance(spec, list) else [spec]
    n = 1 + 1 + 1 + 1                # forces and tile lists; spread; stream-collide; interpolation + advection
    if any(w.lam != 1.0 for w in specs):
        n += 3                       # column reset, face crossings, column sort
    if any(w.volume_correction for w in specs):
        n += 1                       # FP64 volume and centroid, rescale (one cooperative launch)
    return n


GOLDEN64 = os.path.join(ROOT, "tests", "golden", "statics64_oracle.txt")


def run_accuracy_vs_oracle(I, iblb, torch):
    """FP32, FP16 and BF16 storage against the FP64 oracle's stored
    trajectories of the half-scale statics case (64^3, R = 12, L4 mesh,
    xi = 2, volume correction off, theta_eq in {30, 60, 90, 120, 150} deg,
    observed every 1000 steps up to 20000; written from the oracle alone):
    the largest contact-angle difference (eq. angleh with R0 and with the
    volume-equivalent radius, angles below 175 deg) and relative volume
    difference over every observation, all five angles in one batched
    context per storage."""
    stream = torch.cuda.current_stream().cuda_stream
    g = np.loadtxt(GOLDEN64)
    angles = sorted(set(g[:, 0]))
    stops = sorted(set(g[:, 1]))
    out = {"reference": "FP64 oracle, 64^3 half-scale statics, volume correction off", "steps": int(stops[-1]),
           "theta_eq_deg": angles}
    for storage in ("f32", "f16", "bf16"):
        specs = [I.workload_statics_64(th, storage) for th in angles]
        lats = [iblb.lattice_desc(w.nx, w.ny, w.nz, tau_out=w.tau, lam=w.lam, storage=storage) for w in specs]
        phys = [iblb.physics_desc(sigma=w.sigma, theta_eq_deg=w.theta_deg, xi=w.xi, volume_correction=0)
                for w in specs]
        ctx = iblb.iblb_batch_create(lats, phys, stream)
        dth, dv = 0.0, 0.0
        try:
            for k, w in enumerate(specs):
                iblb.iblb_set_membrane(ctx, k, *w.mesh())
            done = 0
            for st in stops:
                iblb.iblb_step(ctx, int(st) - done)
                done = int(st)
                for k, th in enumerate(angles):
                    o = iblb.iblb_observe(ctx, k, 0.05, 0.1)
                    row = g[(g[:, 0] == th) & (g[:, 1] == st)][0]
                    for col, key in ((6, "theta_R0_deg"), (7, "theta_RV_deg")):
                        if row[col] < 175.0:
                            dth = max(dth, abs(o[key] - row[col]))
                    dv = max(dv, abs(o["volume"] / row[2] - 1.0))
        finally:
            iblb.iblb_destroy(ctx)
        out[f"max_abs_dtheta_{storage}_deg"] = dth
        out[f"max_rel_dvolume_{storage}"] = dv
    return out


def run_accuracy(I, iblb, torch, steps, angles=(30.0, 60.0, 90.0, 120.0, 150.0)):
    """Contact angle after `steps` steps of the 128^3 statics droplet for each
    theta_eq, all angles in one batched context per storage; reduced storage
    against FP32 storage on the same GPU."""
    stream = torch.cuda.current_stream().cuda_stream
    res = {}
    for storage in ("f32", "f16", "bf16"):
        specs = [I.workload_statics_128(th, storage) for th in angles]
        lats = [iblb.lattice_desc(w.nx, w.ny, w.nz, tau_out=w.tau, lam=w.lam, storage=storage) for w in specs]
        phys = [iblb.physics_desc(sigma=w.sigma, theta_eq_deg=w.theta_deg, xi=w.xi,
                                  volume_correction=int(w.volume_correction)) for w in specs]
        ctx = iblb.iblb_batch_create(lats, phys, stream)
        try:
            for k, w in enumerate(specs):
                xyz, tri = w.mesh()
                iblb.iblb_set_membrane(ctx, k, xyz, tri)
            iblb.iblb_step(ctx, steps)
            obs = [iblb.iblb_observe(ctx, k) for k in range(len(angles))]
        finally:
            iblb.iblb_destroy(ctx)
        res[storage] = obs
    out = {"steps": steps, "theta_eq_deg": list(angles),
           "theta_RV_deg": {s: [o["theta_RV_deg"] for o in res[s]] for s in res},
           "volume": {s: [o["volume"] for o in res[s]] for s in res}}
    for s in ("f16", "bf16"):
        out[f"max_abs_dtheta_{s}_vs_f32_deg"] = max(abs(a["theta_RV_deg"] - b["theta_RV_deg"])
                                                   for a, b in zip(res[s], res["f32"]))
        out[f"max_rel_dvolume_{s}_vs_f32"] = max(abs(a["volume"] / b["volume"] - 1.0)
                                                for a, b in zip(res[s], res["f32"]))
    return out


LB_SHAPE = {}
IB_SHAPE = {}


def run_gpu(spec, storage, steps, warmup, torch, iblb, flush, autotune=True):
    """Device-timed steps with L2 flushed before each; returns per-phase sums."""
    stream = torch.cuda.current_stream().cuda_stream
    ctx, xyz, tri = make_ctx(iblb, spec, storage, stream)
    try:
        if "mult" in LB_SHAPE:
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_LB_ROW_MULT, LB_SHAPE["mult"])
        if "cells" in LB_SHAPE:
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_LB_GROUP_CELLS, LB_SHAPE["cells"])
        if "bps" in LB_SHAPE:
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_LB_BLOCKS_PER_SM, LB_SHAPE["bps"])
        if "stages" in LB_SHAPE:
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_LB_STAGES, LB_SHAPE["stages"])
        if "fused" in IB_SHAPE:
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_FUSED_IB, IB_SHAPE["fused"])
        if "bps" in IB_SHAPE:
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_IB_BLOCKS_PER_SM, IB_SHAPE["bps"])
        if "pdl" in IB_SHAPE:
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_PDL, IB_SHAPE["pdl"])
        if "split" in IB_SHAPE:
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_SPLIT_LB, IB_SHAPE["split"])
        if "far_bps" in IB_SHAPE:
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_LB_FAR_BLOCKS_PER_SM, IB_SHAPE["far_bps"])
        if "graphs" in IB_SHAPE:
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_GRAPHS, IB_SHAPE["graphs"])
        if autotune and not LB_SHAPE:
            iblb.iblb_autotune(ctx, os.path.join(ROOT, "paper_2503_20605_gb300", "_build", "autotune.txt"))
        def timed(mode, n):
            iblb.iblb_set_option(ctx, iblb.IBLB_OPT_PROFILE, mode)
            for _ in range(warmup):
                flush.zero_()
                iblb.iblb_step(ctx, 1)
            iblb.iblb_sync(ctx)
            iblb.iblb_reset_profile(ctx)
            torch.cuda.synchronize()
            for _ in range(n):
                flush.zero_()
                iblb.iblb_step(ctx, 1)
            iblb.iblb_sync(ctx)
            torch.cuda.synchronize()
            return iblb.iblb_get_profile(ctx)

        # the whole step between two events (the value), every phase between
        # events (the breakdown), and the stream-collide kernel alone between
        # two events (the roofline)
        _, step_ms, n = timed(2, steps)
        phases, phase_step_ms, n_ph = timed(1, steps)
        lb_only, _, n_lb = timed(3, steps)
        iblb.iblb_set_option(ctx, iblb.IBLB_OPT_PROFILE, 0)
        # the same steps back to back in one call (no flush between them:
        # each step streams the populations, larger than L2, through it)
        iblb.iblb_step(ctx, warmup)
        b2b = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        b2b[0].record()
        iblb.iblb_step(ctx, steps)
        b2b[1].record()
        torch.cuda.synchronize()
        b2b_ms = b2b[0].elapsed_time(b2b[1])
        traces = []
        for _ in range(TRACE_STEPS):      # after the timed region: one traced step after each flush
            flush.zero_()
            traces.append(iblb.iblb_trace_step(ctx))
        obs = iblb.iblb_observe(ctx, 0)
        nd = iblb.iblb_info(ctx, 0)["n_drops"]
        infos = [iblb.iblb_info(ctx, k) for k in range(nd)]
    finally:
        iblb.iblb_destroy(ctx)
    return dict(phases=phases, step_ms=step_ms, n=n, n_ph=n_ph, obs=obs, cells=sum(i["cells"] for i in infos),
                nodes=sum(i["n_nodes"] for i in infos), drops=nd, lb_kernel_ms=lb_only["lb"] / n_lb,
                in_step=in_step(traces), b2b_ms=b2b_ms)


TRACE_STEPS = 20


def in_step(traces):
    """Medians over traced steps: each kernel from its first warp past the
    wait on the previous kernel to the next kernel's first start (which
    follows its last exit), the span from the force kernel's start to the end
    of the last kernel, and the membrane's share of it (span minus the
    stream-collide kernel)."""
    names = [k for k in traces[0] if traces[0][k] is not None]
    med = lambda f: statistics.median(f(t) for t in traces)
    out = {k: med(lambda t, k=k: t[k]["end_us"] - t[k]["first_start_us"]) for k in names}
    span = lambda t: max(t[k]["end_us"] for k in names) - t["force"]["first_start_us"]
    out["span"] = med(span)
    out["membrane"] = med(lambda t: span(t) - (t["lb"]["end_us"] - t["lb"]["first_start_us"]))
    out["steps"] = len(traces)
    return out


def extra_workload(name, specs, storage, steps, warmup, torch, iblb, flush, autotune):
    """Throughput line of a further workload (same timing as the headline)."""
    r = run_gpu(specs, storage, steps, warmup, torch, iblb, flush, autotune=autotune)
    KP = r["n_ph"]
    ph = {k: v / KP for k, v in r["phases"].items()}
    ib = ph["forces"] + ph["spread"] + ph["inout"] + ph["advect"] + ph["reduce"]
    bpc = BYTES_PER_CELL[storage]
    return {"workload": name, "storage": storage, "droplets": r["drops"], "cells": r["cells"], "nodes": r["nodes"],
            "value": r["cells"] * r["n"] / (r["step_ms"] * 1e-3) / 1e6, "unit": "MLUPS",
            "ms_per_step": r["step_ms"] / r["n"], "phase_ms_per_step": ph,
            "ib_nodes_per_s": r["nodes"] / (ib * 1e-3),
            "lb_kernel_gbs": r["cells"] * bpc / (r["lb_kernel_ms"] * 1e-3) / 1e9,
            "in_step_us": r["in_step"],
            "ib_nodes_per_s_in_step": r["nodes"] / (r["in_step"]["membrane"] * 1e-6),
            "gpu_launches_per_step": launches_per_step(specs)}


def run_e2e(spec, storage, steps, warmup, torch, iblb):
    """Through the public API with host buffers: each step uploads the node
    positions from pinned host memory, advances one step and reads back the
    node positions and the observables (contact angle, volume, mass)."""
    stream = torch.cuda.current_stream().cuda_stream
    ctx, xyz, tri = make_ctx(iblb, spec, storage, stream)
    try:
        pin = torch.empty((len(xyz), 3), dtype=torch.float64, pin_memory=True)
        host = pin.numpy()
        host[:] = xyz
        for _ in range(warmup):
            iblb.iblb_set_nodes(ctx, 0, host)
            iblb.iblb_step(ctx, 1)
            iblb.iblb_get_nodes(ctx, 0, host)
            iblb.iblb_observe(ctx, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            iblb.iblb_set_nodes(ctx, 0, host)
            iblb.iblb_step(ctx, 1)
            iblb.iblb_get_nodes(ctx, 0, host)
            iblb.iblb_observe(ctx, 0)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        cells = iblb.iblb_info(ctx, 0)["cells"]
    finally:
        iblb.iblb_destroy(ctx)
    n = len(xyz)
    return dict(value=cells * steps / dt / 1e6, unit="MLUPS", h2d_bytes_per_step=n * 3 * 8,
                d2h_bytes_per_step=n * 3 * 8 + 8 + 8 * 15)


def run_mlp(I, iblb, torch):
    """Warm-start network: Adam training steps (batch 256) and inference of
    200 cases, wall-clock around the library calls after a warm-up call."""
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(0)
    x = I.warmstart_cases(2048, 3)
    y = 1.0 + 0.1 * rng.standard_normal((2048, 64))
    m = iblb.iblb_mlp_create(I.mlp_init(0), 256, stream)
    try:
        iblb.iblb_mlp_train(m, x, y, 2, 256, 1e-3, 1)
        torch.cuda.synchronize()
        epochs = 50
        t0 = time.perf_counter()
        iblb.iblb_mlp_train(m, x, y, epochs, 256, 1e-3, 2)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        steps = epochs * (2048 // 256)
        xt = I.warmstart_cases(200, 4)
        iblb.iblb_mlp_predict(m, xt)
        t1 = time.perf_counter()
        for _ in range(20):
            iblb.iblb_mlp_predict(m, xt)
        dp = (time.perf_counter() - t1) / 20
    finally:
        iblb.iblb_mlp_destroy(m)
    flop_fwd = 2 * (3 * 256 + 2 * 256 * 256 + 256 * 64)      # per sample
    flop_step = 3 * flop_fwd * 256                            # forward + backward (two GEMMs per layer)
    return {"train_step_ms": dt / steps * 1e3, "train_tflops": flop_step * steps / dt / 1e12,
            "predict_200_ms": dp * 1e3, "bf16_peak_sustained_tflops": peaks_bf16(),
            "note": "latency-bound: 128 x 256 x 256 tiles, one CTA per 128 rows"}


def peaks_bf16():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)).get("bf16_tflops_sustained")
    return 1700.0


def host_description():
    """Core count and CPU model of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine()}


def cpu_oracle(spec, budget_s, steps_cap, threads=1):
    """The FP64 oracle on the host cores: full steps of the same workload
    until the time budget is used (at least one), its stream-collide loop
    on `threads` threads."""
    import oracle.oracle as O
    O.build()
    O.set_threads(threads)
    xyz, tri = spec.mesh()
    A = O.wetting_A(spec.sigma, math.radians(spec.theta_deg), spec.xi)
    s = O.Sim(O.make_params(spec.nx, spec.ny, spec.nz, tau_out=spec.tau, tau_in=spec.tau_in, sigma=spec.sigma,
                            wetting=1, A=A, xi=spec.xi, volume_correction=int(spec.volume_correction)))
    s.set_membrane(xyz, tri)
    t0 = time.perf_counter()
    n = 0
    while n < steps_cap and (n == 0 or time.perf_counter() - t0 < budget_s):
        s.step(1)
        n += 1
    dt = time.perf_counter() - t0
    return n, dt, s.cells, len(xyz)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f16", choices=["f16", "bf16", "f32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--only-main", action="store_true",
                    help="time only the headline storage (no FP32 line, no e2e loop); for profiler runs")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--lb-row-mult", type=int, default=0,
                    help="stream-collide rows per group multiple (implies --no-autotune)")
    ap.add_argument("--fused-ib", type=int, default=-1, help="1/0: cooperative or separate membrane kernels")
    ap.add_argument("--split-lb", type=int, default=-1, help="1/0: far stream-collide groups on a second stream")
    ap.add_argument("--pdl", type=int, default=-1, help="1/0: programmatic dependent launch in the step")
    ap.add_argument("--graphs", type=int, default=-1, help="1/0: replay captured graphs or launch eagerly")
    ap.add_argument("--lb-far-blocks-per-sm", type=int, default=-1, help="blocks per SM of the far groups")
    ap.add_argument("--ib-blocks-per-sm", type=int, default=-1, help="blocks per SM of the cooperative kernels")
    ap.add_argument("--lb-group-cells", type=int, default=0,
                    help="about this many cells per stream-collide group (implies --no-autotune)")
    ap.add_argument("--lb-stages", type=int, default=0,
                    help="stream-collide pipeline stages 2..8 (implies --no-autotune)")
    ap.add_argument("--lb-blocks-per-sm", type=int, default=-1,
                    help="stream-collide blocks per SM, 0 = as many as fit (implies --no-autotune)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the spreading (256x256x128, lambda=10, BF16) and 64-droplet batch lines")
    ap.add_argument("--accuracy-steps", type=int, default=20000,
                    help="steps of the FP16/BF16-vs-FP32 contact-angle comparison at 128^3 (0: skip)")
    args = ap.parse_args()

    from paper_2503_20605_gb300 import inputs as I
    if args.lb_row_mult > 0:
        LB_SHAPE["mult"] = args.lb_row_mult
    if args.lb_group_cells > 0:
        LB_SHAPE["cells"] = args.lb_group_cells
    if args.lb_blocks_per_sm >= 0:
        LB_SHAPE["bps"] = args.lb_blocks_per_sm
    if args.lb_stages > 0:
        LB_SHAPE["stages"] = args.lb_stages
    if args.fused_ib >= 0:
        IB_SHAPE["fused"] = args.fused_ib
    if args.ib_blocks_per_sm >= 0:
        IB_SHAPE["bps"] = args.ib_blocks_per_sm
    if args.pdl >= 0:
        IB_SHAPE["pdl"] = args.pdl
    if args.split_lb >= 0:
        IB_SHAPE["split"] = args.split_lb
    if args.graphs >= 0:
        IB_SHAPE["graphs"] = args.graphs
    if args.lb_far_blocks_per_sm >= 0:
        IB_SHAPE["far_bps"] = args.lb_far_blocks_per_sm
    spec = I.workload_statics_128(90.0, args.storage)
    rank, world, local = dist_env()
    workload = "statics droplet 128^3 (D3Q19 tau=1, walls z, L5 icosphere 10242 nodes, R=24, sigma=0.005, " \
               "xi=2.4, theta_eq=90, volume correction)"

    if args.impl == "reference":
        if rank != 0:
            return
        cores = os.cpu_count() or 1
        n, dt, cells, nodes = cpu_oracle(spec, budget_s=120.0, steps_cap=max(1, args.steps + args.warmup),
                                         threads=cores)
        v = cells * n / dt / 1e6
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / n * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload, "storage": "f64 (oracle)", "cells": cells, "nodes": nodes},
                "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                 "sample": f"{n} full oracle steps of the workload (time budget 120 s), "
                                           f"stream-collide loop on {cores} threads",
                                 "host": host_description()},
                "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2503_20605_gb300 import iblb
    iblb.lib()

    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    barrier()
    with Clocks(local) as clk:
        main_run = run_gpu(spec, args.storage, args.steps, args.warmup, torch, iblb, flush,
                           autotune=not args.no_autotune)
    barrier()
    run32, e2e = None, None
    if not args.only_main:
        spec32 = I.workload_statics_128(90.0, "f32")
        run32 = run_gpu(spec32, "f32", args.steps, args.warmup, torch, iblb, flush, autotune=not args.no_autotune)
        e2e = run_e2e(spec, args.storage, max(20, args.steps // 4), 3, torch, iblb)

    step_ms = max_over_ranks(main_run["step_ms"], world, "cuda")
    K = main_run["n"]
    cells, nodes = main_run["cells"], main_run["nodes"]
    value = whole_job_mlups(cells, K, step_ms, world)
    ph = main_run["phases"]
    KP = main_run["n_ph"]
    ib_ms = (ph["forces"] + ph["spread"] + ph["inout"] + ph["advect"] + ph["reduce"]) / KP   # per step
    lb_ms = main_run["lb_kernel_ms"]          # the stream-collide kernel between two events of its own
    peak, src = peaks()
    bpc = BYTES_PER_CELL[args.storage]
    achieved = cells * bpc / (lb_ms * 1e-3) / 1e9
    traffic = ncu_traffic(args.storage)
    fp32 = None
    if run32:
        ph32 = run32["phases"]
        KP32 = run32["n_ph"]
        ib32 = (ph32["forces"] + ph32["spread"] + ph32["inout"] + ph32["advect"] + ph32["reduce"]) / KP32
        lb32 = run32["lb_kernel_ms"]
        fp32 = {"value": cells * run32["n"] / (run32["step_ms"] * 1e-3) / 1e6, "unit": "MLUPS",
                "ms_per_step": run32["step_ms"] / run32["n"],
                "phase_ms_per_step": {k: v / KP32 for k, v in ph32.items()},
                "ib_nodes_per_s": nodes / (ib32 * 1e-3),
                "lb_kernel_gbs": cells * BYTES_PER_CELL["f32"] / (lb32 * 1e-3) / 1e9,
                "theta_RV_deg_after": run32["obs"]["theta_RV_deg"]}

    extra = None
    if not args.only_main and not args.no_extra:
        extra = [
            extra_workload("spreading droplet 256x256x128 (tau_out=0.8, lambda=10, L6 icosphere 40962 nodes, R=40, "
                           "theta_eq=20, sigma=0.005, xi=2)", I.workload_spreading_256("bf16"), "bf16",
                           max(20, args.steps // 2), args.warmup, torch, iblb, flush, not args.no_autotune),
            extra_workload("batch of 64 droplets (sides U{48..96}, R U[6,20], theta_eq U[20,160], tau U[0.6,1.2], "
                           "sigma=0.01, seed 2025)", I.workload_batch(64, 2025, "f16"), "f16",
                           max(20, args.steps // 2), args.warmup, torch, iblb, flush, not args.no_autotune)]

    mlp = None
    if rank == 0 and not args.only_main:
        mlp = run_mlp(I, iblb, torch)

    accuracy = None
    if rank == 0 and not args.only_main and args.accuracy_steps > 0:
        accuracy = {"vs_oracle_64": run_accuracy_vs_oracle(I, iblb, torch),
                    "vs_f32_128": run_accuracy(I, iblb, torch, args.accuracy_steps)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        host = host_description()
        allc = host["nproc"] or 1
        n1, dt1, c_cells, c_nodes = cpu_oracle(spec, args.cpu_budget / 2, 1000, threads=1)
        na, dta, _, _ = cpu_oracle(spec, args.cpu_budget / 2, 1000, threads=allc)
        cpu = {"value": c_cells * na / dta / 1e6, "unit": "MLUPS", "cores": allc, "kind": "oracle",
               "sample": f"{na} full FP64 oracle steps of the same 128^3 workload with the stream-collide loop "
                         f"on {allc} threads; {n1} steps on one thread",
               "one_core": {"value": c_cells * n1 / dt1 / 1e6, "unit": "MLUPS",
                            "ib_nodes_per_s": c_nodes * n1 / dt1},
               "all_cores_ib_nodes_per_s": c_nodes * na / dta, "host": host}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": step_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "storage": args.storage, "cells": cells, "nodes": nodes,
                       "grid": [spec.nx, spec.ny, spec.nz], "l2": "flushed (512 MB write) before every timed step",
                       "parallelism": f"replicas x{world}"},
            "ib_nodes_per_s": world * nodes / (ib_ms * 1e-3),
            # its fraction of an HBM bound: 64 stencil cells x 24 B (a read
            # of U and a write of F, 3 x FP32 each) per node at the measured
            # copy bandwidth
            "ib_roofline": {"bound_nodes_per_s": peak * 1e9 / (64 * 24),
                            "frac": world * nodes / (ib_ms * 1e-3) / (peak * 1e9 / (64 * 24)),
                            "peak_gbs": peak, "peak_source": src},
            "phase_ms_per_step": {k: v / KP for k, v in ph.items()},
            "fp32": fp32,
            # per-warp %globaltimer stamps of steps traced after the timed
            # region (iblb_trace_step, L2 flushed before each): every kernel
            # from its first warp past the wait on the previous kernel to the
            # next kernel's first start, as it runs inside the chained step
            "in_step": {
                "us": {k: v for k, v in main_run["in_step"].items() if k != "steps"},
                "steps": main_run["in_step"]["steps"],
                "ib_nodes_per_s": world * nodes / (main_run["in_step"]["membrane"] * 1e-6),
                "lb_achieved_gbs": cells * bpc / (main_run["in_step"]["lb"] * 1e-6) / 1e9,
                "lb_frac": cells * bpc / (main_run["in_step"]["lb"] * 1e-6) / 1e9 / peak,
            },
            "back_to_back": {
                "value": whole_job_mlups(cells, K, max_over_ranks(main_run["b2b_ms"], world, "cuda"), world),
                "unit": "MLUPS", "ms_per_step": main_run["b2b_ms"] / K,
                "l2": "not flushed: the K steps in one iblb_step call; every step streams the populations "
                      "(larger than L2) through it"},
            "roofline": {"bound": "hbm", "kernel": "lb_kernel (fused stream-collide)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": src,
                         "algorithmic_bytes_per_cell": bpc, "traffic": traffic},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_step(spec) * K,
            "clocks": clk.summary(),
            "theta_RV_deg_after": main_run["obs"]["theta_RV_deg"],
            "accuracy": accuracy,
            "other_workloads": extra,
            "warmstart_mlp": mlp,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
