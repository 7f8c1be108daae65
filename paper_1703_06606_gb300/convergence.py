"""Self-convergence study of Sec. 9 (Table 1) and the per-step cost of Table 2.

The convergence test of Sec. 9 refines the grid and the time step together
(m = 16, 32, ..., dt = 16 h^2) from c = cos(2 pi x) + cos(2 pi y), and compares
each solution with the next finer one after pushing the coarse solution up to
the fine grid: the L2 norm of the difference, and the rate log2(e_{2h}/e_h).
With dt proportional to h^2 the first-order time error is O(h^2), so the rate
tends to 2.  The push-up is the cell-centred bilinear interpolation (weights
9/16, 3/16, 3/16, 1/16, mirror at the walls): piecewise-constant injection
would add an O(h) interpolation error and cap the rate at 1.

    python -m paper_1703_06606_gb300.convergence --m 16 32 64 128 256

The solver class is a parameter (`run(solver_cls, ...)`): any class with the
qnsch.Solver interface (set_fields, step, get_fields).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import workloads


def prolong_bilinear(a):
    """Cell-centred bilinear interpolation of an (m2, m1) cell field onto the
    (2 m2, 2 m1) grid of half the spacing; the ghost row/column mirrors the
    boundary cell (homogeneous Neumann)."""
    m2, m1 = a.shape
    p = np.pad(a, 1, mode="edge")
    out = np.empty((2 * m2, 2 * m1))
    for dj in (0, 1):
        sj = -1 if dj == 0 else 1
        for di in (0, 1):
            si = -1 if di == 0 else 1
            c = p[1:m2 + 1, 1:m1 + 1]
            cx = p[1:m2 + 1, 1 + si:m1 + 1 + si]
            cy = p[1 + sj:m2 + 1 + sj, 1:m1 + 1]
            cxy = p[1 + sj:m2 + 1 + sj, 1 + si:m1 + 1 + si]
            out[dj::2, di::2] = (9.0 * c + 3.0 * cx + 3.0 * cy + cxy) / 16.0
    return out


def l2_cells(a, h):
    """(h^2 sum a^2)^(1/2) over the cells."""
    return math.sqrt(h * h * float(np.sum(a * a)))


def solve(solver_cls, m, **options):
    """Run the Sec. 9 workload on level m to t = 1/16; returns (fields, dict)."""
    P = workloads.convergence_test(m)
    s = solver_cls(**P.create_kwargs(), tol=P.tol, maxcyc=100, **options)
    s.set_fields(P.fields())
    cyc = []
    t0 = time.perf_counter()
    for _ in range(P.steps):
        n, _ = s.step(P.dt)
        cyc.append(n)
    sec = time.perf_counter() - t0
    f = s.get_fields()
    close = getattr(s, "close", None)
    if close:
        close()
    return f, {"m": m, "steps": P.steps, "dt": P.dt, "vcycles_per_step": float(np.mean(cyc)),
               "seconds": sec, "s_per_step": sec / P.steps}


def run(solver_cls, ms=(16, 32, 64, 128, 256), field="c", **options):
    """The Table 1 study: for consecutive levels (m/2, m) the L2 difference of
    `field` between the level-m solution and the pushed-up level-m/2 solution,
    and the rate."""
    rows, prev_f, prev_e = [], None, None
    for m in ms:
        f, info = solve(solver_cls, m, **options)
        if prev_f is not None:
            e = l2_cells(f[field] - prolong_bilinear(prev_f[field]), 1.0 / m)
            info["pair"] = "%d & %d" % (m // 2, m)
            info["error"] = e
            info["rate"] = math.log2(prev_e / e) if prev_e else None
            prev_e = e
        rows.append(info)
        prev_f = f
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, nargs="+", default=[16, 32, 64, 128, 256])
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--coupled", type=int, default=0)
    ap.add_argument("--scheme", type=int, default=0)
    a = ap.parse_args()
    from . import qnsch
    for row in run(qnsch.Solver, a.m, precision=a.precision, coupled=a.coupled, scheme=a.scheme):
        print(json.dumps(row))


if __name__ == "__main__":
    main()
