"""Autotuner for the launch-shape options of libqnsch.so.

The kernels' launch shapes are chosen per level by thresholds (include/qnsch.h):
how many cells per colour a level may have for its Vanka, coupled or CH blocks
to run with four lanes per block (vanka_team_max, ch_team_max and their FP32
counterparts), from which size the coarse levels run as one single-block
V-cycle (fuse_cells, fuse_cells32), and from which size the error-equation
levels smooth as one banded wavefront launch and with what band height, its
tile shape (wave_cells32, wave_rows), or in the skewed-chunk schedule and with
what chunk height (skew_cells32, skew_rows).  It also searches the smoothing counts
(nu1, nu2, nu_coarse), which trade the cost of a V-cycle against the number
of V-cycles a step needs.  The best values depend on the grid, the
precision and the smoother, and on how busy the GPU is.  This module picks
them by measurement: coordinate descent over the thresholds of the workload's
precision, timing whole time steps from the same initial state, and keeps the
result in a JSON table keyed by GPU, grid, precision and smoother.

    python -m paper_1703_06606_gb300.autotune --workload drop --precision 1 \\
        --coupled 1 --table tuned.json

serve.Server(tuned_table=...) applies a table's entries to the instances it
admits.  Options never change the fixed point of a step (the discrete
solution at the tolerance), only the order in which per-lane sums are added,
which kernels run and, for the smoothing counts, the path of the iteration.
"""
from __future__ import annotations

import argparse
import json
import os
import time

# candidate values per option; the first is the library default
CANDIDATES = {
    "vanka_team_max": [8192, 2048, 32768, 0],
    # eight lanes per FP64 Vanka block up to this many cells per colour (0: never)
    "vanka_team8_max": [0, 2048, 512],
    # a lane pair per FP64 Vanka block above vanka_team_max, up to this many
    # cells per colour (0: never)
    "vanka_pair_max": [0, 1 << 20, 8192],
    # single-lane FP64 Vanka launches split between one lane per block and
    # lane pairs (0: never, 1: by the cost model)
    "vanka_split": [0, 1],
    # the fused coarse V-cycle of the FP64 levels on a shared-memory copy (1) or
    # from global memory (0)
    "coarse_smem": [1, 0],
    "ch_team_max": [4096, 0, 16384],
    "fuse_cells": [128, 32, 512, 4096],
    "vanka_team_max32": [65536, 0, 8192, 131072, 1 << 30],
    "ch_team_max32": [0, 4096],
    "fuse_cells32": [512, 128, 2048],
    # blocks of the fused V-cycle's launch (1, or one thread-block cluster)
    "fuse_ctas": [1, 16, 4],
    # the banded wavefront on the error-equation levels: from which level size
    # (0: never) and with how many rows per band (its tile height)
    "wave_cells32": [0, 1 << 20, 1 << 16],
    "wave_rows": [8, 4, 16, 32],
    # the skewed-chunk schedule on the error-equation levels: from which level
    # size (0: never) and with chunks of how many rows
    "skew_cells32": [0, 1 << 20, 1 << 17],
    "skew_rows": [32, 64, 16],
    # smoothing steps before and after the coarse-grid correction, and on the
    # coarsest grid (more steps: fewer, dearer V-cycles)
    "nu1": [2, 3, 1],
    "nu2": [2, 3, 1],
    "nu_coarse": [4, 2, 8],
    # the finest level's own smoothing counts (-1: nu1, nu2)
    "nu1_fine": [-1, 2, 3],
    "nu2_fine": [-1, 3, 2],
}
# a candidate's steps are cut off at this multiple of the best time per step
CUTOFF = 20.0
# a candidate replaces the incumbent only if it is at least this much faster
# (relative), so that timing noise does not move a knob
MIN_GAIN = 0.005
# the options that shape the launches of each precision (0 FP64, 1 mixed,
# 2 FP64 error form: its error levels use the FP64 thresholds)
KNOBS = {
    0: ["vanka_team_max", "vanka_team8_max", "vanka_pair_max", "vanka_split", "ch_team_max",
        "fuse_cells", "fuse_ctas", "coarse_smem", "nu1", "nu2", "nu_coarse", "nu1_fine",
        "nu2_fine"],
    1: ["vanka_team_max32", "ch_team_max32", "fuse_cells32", "fuse_ctas", "wave_cells32",
        "wave_rows", "skew_cells32", "skew_rows", "nu1", "nu2", "nu_coarse", "nu1_fine", "nu2_fine"],
    2: ["vanka_team_max32", "ch_team_max32", "fuse_cells", "fuse_ctas", "wave_cells32",
        "wave_rows", "skew_cells32", "skew_rows", "nu1", "nu2", "nu_coarse", "nu1_fine", "nu2_fine"],
}


def key_of(P, precision, coupled, scheme, device=""):
    """Table key: device name, grid, boundary, precision and smoother."""
    return "%s|%dx%d|px%d|p%d|c%d|s%d" % (device, P.m1, P.m2, int(P.periodic_x), precision,
                                          coupled, scheme)


def _cuda_clock():
    import torch
    torch.cuda.synchronize()
    return time.perf_counter()


def time_steps(solver_cls, P, options, steps, warmup, clock):
    """Seconds per time step of the workload under `options`, from its initial
    state, after `warmup` steps; None if a step fails."""
    s = solver_cls(**P.create_kwargs(), tol=P.tol, **options)
    try:
        s.set_fields(P.fields())
        for _ in range(warmup):
            s.step(P.dt)
        t0 = clock()
        for _ in range(steps):
            s.step(P.dt)
        return (clock() - t0) / steps
    except Exception:
        return None
    finally:
        close = getattr(s, "close", None)
        if close:
            close()


def tune(P, precision=0, coupled=0, scheme=0, steps=4, warmup=2, solver_cls=None, clock=None,
         candidates=None, rounds=2):
    """Coordinate descent over the launch-shape options of `precision`: each
    option in turn takes the candidate value with the shortest time per step,
    the others held, for `rounds` passes or until nothing changes.  Returns
    (best options, best seconds per step, every (options, seconds) measured)."""
    if solver_cls is None:
        from . import qnsch
        solver_cls = qnsch.Solver
    clock = clock or _cuda_clock
    cand = dict(CANDIDATES, **(candidates or {}))
    base = {"precision": precision, "coupled": coupled, "scheme": scheme}
    best = {k: cand[k][0] for k in KNOBS[precision]}
    seen = {}

    def measure(opts):
        key = tuple(sorted(opts.items()))
        if key not in seen:
            # once a time is known, a candidate whose step takes 20 times as
            # long is cut off by the step's time limit (QNSCH_ETIMEOUT) and
            # counts as failed, so one pathological shape cannot stall the search
            cap = {} if best_t is None else {"step_time_limit": max(CUTOFF * best_t, 2.0)}
            seen[key] = time_steps(solver_cls, P, dict(base, **opts, **cap), steps, warmup,
                                   clock)
        return seen[key]

    best_t = None
    best_t = measure(best)
    for _ in range(rounds):
        changed = False
        for k in KNOBS[precision]:
            for v in cand[k]:
                if v == best[k]:
                    continue
                trial = dict(best, **{k: v})
                t = measure(trial)
                if t is not None and (best_t is None or t < best_t * (1.0 - MIN_GAIN)):
                    best, best_t, changed = trial, t, True
        if not changed:
            break
    history = [(dict(k), t) for k, t in seen.items()]
    return best, best_t, history


def load_table(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_entry(path, key, options, seconds):
    """Add or replace one entry of the JSON table at `path`."""
    table = load_table(path)
    table[key] = {"options": options, "ms_per_step": None if seconds is None else seconds * 1e3}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(table, P, precision, coupled, scheme, device=""):
    """The tuned options of a workload, or {} when the table has none."""
    e = table.get(key_of(P, precision, coupled, scheme, device))
    return dict(e["options"]) if e else {}


def device_name():
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return ""


def main():
    from . import workloads
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="drop", choices=["drop", "capillary", "rt"])
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--coupled", type=int, default=0)
    ap.add_argument("--scheme", type=int, default=0)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--table", default="qnsch_tuned.json")
    a = ap.parse_args()
    P = {"drop": workloads.rising_drop_256x512, "capillary": workloads.capillary_64,
         "rt": workloads.rayleigh_taylor_1024x4096}[a.workload]()
    best, t, hist = tune(P, a.precision, a.coupled, a.scheme, steps=a.steps)
    for opts, sec in sorted(hist, key=lambda x: (x[1] is None, x[1] or 0)):
        print(json.dumps(opts), "ms/step", None if sec is None else round(sec * 1e3, 3))
    save_entry(a.table, key_of(P, a.precision, a.coupled, a.scheme, device_name()), best, t)
    print("best", json.dumps(best), "ms/step", None if t is None else round(t * 1e3, 3))


if __name__ == "__main__":
    main()
