"""Checkpoint and resume of one simulation (host side; `.npz` files).

The state of an instance between time steps is its committed fields c^n, mu^n,
u^n, v^n, p^n (mu and p only as the next step's initial guesses, but keeping
them makes a resumed run repeat the uninterrupted one bit for bit), the
parameters it was created with, its solver options, and the time t and step
count n the caller keeps.  save() writes them to one .npz file (atomically:
a temporary file renamed into place); load() reads and checks it.

    from paper_1703_06606_gb300 import qnsch
    s.save_checkpoint("run.npz", t=t, n=n)
    s, t, n = qnsch.Solver.from_checkpoint("run.npz")
"""
from __future__ import annotations

import json
import os

import numpy as np

FORMAT = 1
FIELDS = ("c", "mu", "u", "v", "p")
# the parameters of qnsch_create, as the Solver takes them
PARAMS = ("m1", "m2", "Lx", "periodic_x", "levels", "rho1", "rho2", "eta1", "eta2", "Re", "We",
          "Pe", "Cn", "Fr")
# per-handle options that change a step's arithmetic or its control ("pdl" is
# process-wide and not part of an instance's state); scheme first, then
# precision and coupled, so that restoring them in this order never meets a
# forbidden combination on the way
OPTIONS = ("scheme", "precision", "coupled", "nu1", "nu2", "nu_coarse", "maxcyc", "tol",
           "omega_vanka", "M", "eta_st", "eps_mob", "graphs", "fuse_cells", "fuse_cells32",
           "vanka_team_max", "ch_team_max", "vanka_team_max32", "ch_team_max32",
           "step_time_limit", "diverge_cycles", "device_loop", "wave_cells32", "wave_rows",
           "vanka_team8_max", "vanka_pair_max", "vanka_split", "coarse_smem", "skew_cells32", "skew_rows", "predictor", "nu1_fine", "nu2_fine",
           "fuse_ctas")


def field_shapes(m1, m2):
    """(rows, columns) of each field in the host layout of qnsch_get_fields:
    cells m2 x m1, u on all x-edges m2 x (m1 + 1), v on all y-edges
    (m2 + 1) x m1."""
    return {"c": (m2, m1), "mu": (m2, m1), "p": (m2, m1), "u": (m2, m1 + 1), "v": (m2 + 1, m1)}


def save(path, fields, params, options, t=0.0, n=0, library=None, history=()):
    """Write one checkpoint.  fields: the five arrays; params: the creation
    parameters (PARAMS); options: option key -> value; library: the version of
    the library that computed the state (recorded, not checked on load);
    history: the earlier states the option "predictor" extrapolates from, as
    (fields, dt) pairs, the most recent first (qnsch_get_history)."""
    missing = [k for k in PARAMS if k not in params]
    if missing:
        raise ValueError("checkpoint parameters missing: %s" % missing)
    shapes = field_shapes(int(params["m1"]), int(params["m2"]))
    arrays = {}
    for k in FIELDS:
        a = np.ascontiguousarray(fields[k], dtype=np.float64)
        if a.shape != shapes[k]:
            raise ValueError("field %s has shape %s, expected %s" % (k, a.shape, shapes[k]))
        arrays[k] = a
    hdt = []
    for j, (hf, dt) in enumerate(history):
        for k in FIELDS:
            a = np.ascontiguousarray(hf[k], dtype=np.float64)
            if a.shape != shapes[k]:
                raise ValueError("history %d field %s has shape %s, expected %s"
                                 % (j, k, a.shape, shapes[k]))
            arrays["h%d_%s" % (j, k)] = a
        hdt.append(float(dt))
    meta = {"format": FORMAT, "params": {k: params[k] for k in PARAMS},
            "options": {k: float(v) for k, v in options.items()}, "t": float(t), "n": int(n),
            "library": None if library is None else list(library), "history_dt": hdt}
    tmp = "%s.tmp%d" % (path, os.getpid())
    with open(tmp, "wb") as f:
        np.savez(f, meta=np.array(json.dumps(meta)), **arrays)
    os.replace(tmp, path)


def load(path):
    """Read a checkpoint: (fields, params, options, t, n).  Raises ValueError
    for an unknown format or fields of the wrong shape."""
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(str(z["meta"]))
        if meta.get("format") != FORMAT:
            raise ValueError("unknown checkpoint format %r" % meta.get("format"))
        params = meta["params"]
        shapes = field_shapes(int(params["m1"]), int(params["m2"]))
        fields = {}
        for k in FIELDS:
            a = np.array(z[k], dtype=np.float64)
            if a.shape != shapes[k]:
                raise ValueError("field %s has shape %s, expected %s" % (k, a.shape, shapes[k]))
            fields[k] = a
    opts = {k: meta["options"][k] for k in OPTIONS if k in meta["options"]}
    return fields, params, opts, meta["t"], meta["n"]


def load_history(path):
    """The earlier states a checkpoint recorded, as (fields, dt) pairs, the
    most recent first ([] for a checkpoint without them)."""
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(str(z["meta"]))
        shapes = field_shapes(int(meta["params"]["m1"]), int(meta["params"]["m2"]))
        out = []
        for j, dt in enumerate(meta.get("history_dt", [])):
            f = {}
            for k in FIELDS:
                a = np.array(z["h%d_%s" % (j, k)], dtype=np.float64)
                if a.shape != shapes[k]:
                    raise ValueError("history %d field %s has shape %s" % (j, k, a.shape))
                f[k] = a
            out.append((f, float(dt)))
    return out
