"""Run one simulation: time steps with a per-step JSON-lines log and periodic
checkpoints, from a workload's initial state or from a checkpoint.

    python -m paper_1703_06606_gb300.run --workload drop --steps 100 \\
        --log drop.jsonl --checkpoint drop.npz --every 20
    python -m paper_1703_06606_gb300.run --resume drop.npz --steps 100 \\
        --log drop.jsonl --checkpoint drop.npz --every 20

Each log line records one committed step: its index and time, the V-cycles it
took and its final residual, the mass sums h^2 sum rho and h^2 sum rho c
(Thm. 6.1), the discrete energy and the step's dissipation (Thm. 6.2), and
the wall time of the step.  A failed step (not converged, non-finite, past its
time limit) is logged with its status; the state stays at the last committed
step, which is checkpointed before the error is raised.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

from . import qnsch, workloads


def step_record(solver, n, t, vcycles, residual, wall_ms):
    """The log line of committed step n (time t after it)."""
    m_rho, m_rhoc = solver.mass()
    E, D = solver.energy()
    return {"step": int(n), "t": float(t), "vcycles": int(vcycles), "residual": float(residual),
            "mass_rho": m_rho, "mass_rhoc": m_rhoc, "energy": E, "dissipation": D,
            "wall_ms": float(wall_ms), "status": 0}


def simulate(solver, dt, steps, t=0.0, n=0, log=None, checkpoint=None, every=0,
             clock=time.perf_counter):
    """Advance `solver` by `steps` steps of size dt from time t, step count n.
    log: a text file that receives one JSON line per step; checkpoint: a path
    written every `every` steps (0: only at the end) and at the end.  Returns
    (t, n).  A failing step is logged with its status, the last committed
    state checkpointed, and the error raised."""
    def save():
        if checkpoint:
            solver.save_checkpoint(checkpoint, t=t, n=n)

    for _ in range(steps):
        t0 = clock()
        try:
            cyc, res = solver.step(dt)
        except qnsch.QnschError as e:
            if log is not None:
                log.write(json.dumps({"step": n + 1, "t": t + dt, "status": e.code,
                                      "wall_ms": (clock() - t0) * 1e3}) + "\n")
                log.flush()
            save()
            raise
        wall = (clock() - t0) * 1e3
        t, n = t + dt, n + 1
        if log is not None:
            log.write(json.dumps(step_record(solver, n, t, cyc, res, wall)) + "\n")
            log.flush()
        if every and n % every == 0:
            save()
    save()
    return t, n


WORKLOADS = {"drop": "rising_drop_256x512", "capillary": "capillary_64",
             "rt": "rayleigh_taylor_1024x4096", "small": "small_case"}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="drop", choices=sorted(WORKLOADS))
    ap.add_argument("--config", default=None,
                    help="a JSON problem (workloads.Problem.to_json) instead of --workload")
    ap.add_argument("--resume", default=None, help="checkpoint to start from")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--dt", type=float, default=None, help="default: the workload's")
    ap.add_argument("--precision", type=int, default=None, choices=[0, 1, 2])
    ap.add_argument("--coupled", type=int, default=None, choices=[0, 1])
    ap.add_argument("--scheme", type=int, default=None, choices=[0, 1])
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--step-time-limit", type=float, default=None,
                    help="seconds; a longer step fails with QNSCH_ETIMEOUT")
    ap.add_argument("--diverge-cycles", type=int, default=None,
                    help="stop a step whose residual grew over this many cycles")
    ap.add_argument("--log", default=None, help="JSON-lines step log (appended)")
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--every", type=int, default=0)
    a = ap.parse_args(argv)
    if a.config:
        with open(a.config) as f:
            P = workloads.Problem.from_json(f.read())
    else:
        P = getattr(workloads, WORKLOADS[a.workload])()
    over = {k: v for k, v in (("scheme", a.scheme), ("precision", a.precision),
                              ("coupled", a.coupled), ("tol", a.tol),
                              ("step_time_limit", a.step_time_limit),
                              ("diverge_cycles", a.diverge_cycles)) if v is not None}
    if a.resume:
        s, t, n = qnsch.Solver.from_checkpoint(a.resume, **over)
    else:
        s = qnsch.Solver(**P.create_kwargs(), **dict({"tol": P.tol}, **over))
        s.set_fields(P.fields())
        t, n = 0.0, 0
    log = open(a.log, "a") if a.log else None
    try:
        t, n = simulate(s, a.dt or P.dt, a.steps, t, n, log, a.checkpoint, a.every)
    finally:
        if log:
            log.close()
    print(json.dumps({"t": t, "steps": n}), file=sys.stdout)


if __name__ == "__main__":
    main()
