"""Diagnostics log of a running context: one JSON line per droplet and
interval with the observables of Sec. III and App. C, as the library's
FP64 reductions compute them (mass, enclosed volume and its ratio to the
first observation, area, lowest and highest node, the half-height l of
eq. ell, the contact angle of eq. angleh with R0 and with the current
volume-equivalent radius, the contact radius by protocols (i) and (ii),
and the droplet's device status).

Argument marshalling and bookkeeping only: the steps and the observables
run in libiblb through the C ABI.

    from paper_2503_20605_gb300 import monitor
    monitor.run_logged(ctx, n_steps=20000, every=500, path="drop.jsonl")
"""
from __future__ import annotations

import json

from . import iblb

FIELDS = ("mass", "volume", "area", "zmin", "zmax", "theta_R0_deg", "theta_RV_deg", "rc_cut", "rc_flat",
          "n_cut", "chi_flat", "clamped", "status")


def record(step, k, obs, v0):
    """One log line (a dict) for droplet k at `step` from an observation
    dict of iblb_observe_all; v0 is that droplet's first observed volume."""
    r = {"step": int(step), "droplet": int(k)}
    r.update({f: obs[f] for f in FIELDS})
    r["ell"] = 0.5 * (obs["zmax"] - obs["zmin"])
    r["volume_ratio"] = obs["volume"] / v0 if v0 else None
    return r


def run_logged(ctx, n_steps, every, path, zcut_frac=0.05, eps_flat=0.1, stop_on_error=True,
               step=None, observe_all=None):
    """Advance ctx by n_steps in chunks of `every`, appending a line per
    droplet to the JSONL file at `path` before the first chunk and after
    each one.  Returns the list of records.  A droplet whose status is not
    IBLB_OK ends the run after its line is written when stop_on_error is
    set (the status is logged either way).  `step` and `observe_all`
    default to the library calls."""
    if every <= 0 or n_steps < 0:
        raise ValueError("every must be positive and n_steps non-negative")
    step = step or iblb.iblb_step
    observe_all = observe_all or (lambda c: iblb.iblb_observe_all(c, zcut_frac, eps_flat))
    out, v0, done = [], {}, 0
    with open(path, "a") as fh:
        while True:
            bad = False
            for k, o in enumerate(observe_all(ctx)):
                v0.setdefault(k, o["volume"])
                r = record(done, k, o, v0[k])
                fh.write(json.dumps(r) + "\n")
                out.append(r)
                bad |= o["status"] != iblb.IBLB_OK
            fh.flush()
            if (bad and stop_on_error) or done >= n_steps:
                return out
            n = min(every, n_steps - done)
            step(ctx, n)
            done += n
