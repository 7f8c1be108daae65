"""The autotuner's search and its table, on CPU: a stand-in solver whose time
per step is a known function of the launch-shape options, on a fake clock."""
import pytest

from paper_1703_06606_gb300 import autotune
from paper_1703_06606_gb300 import workloads as W


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def make_solver(clock, cost, calls):
    class FakeSolver:
        def __init__(self, **kw):
            self.kw = kw
            calls.append(kw)

        def set_fields(self, f):
            pass

        def step(self, dt):
            clock.t += cost(self.kw)
            return 5, 1e-10

        def close(self):
            pass
    return FakeSolver


def test_coordinate_descent_finds_the_separable_optimum():
    """cost = sum of per-option penalties: one pass of coordinate descent lands
    on the best candidate of every option, and every trial keeps the workload's
    precision and smoother."""
    clock, calls = FakeClock(), []
    best_of = {"vanka_team_max32": 8192, "ch_team_max32": 4096, "fuse_cells32": 2048}

    def cost(kw):
        return 1.0 + sum(0.0 if kw[k] == v else 0.1 for k, v in best_of.items())
    P = W.small_case(32, 32, False)
    best, t, hist = autotune.tune(P, precision=1, coupled=1, steps=3, warmup=1,
                                  solver_cls=make_solver(clock, cost, calls), clock=clock)
    assert {k: best[k] for k in best_of} == best_of
    assert all(best[k] == autotune.CANDIDATES[k][0] for k in best if k not in best_of)
    assert t == pytest.approx(1.0)
    assert all(c["precision"] == 1 and c["coupled"] == 1 and c["scheme"] == 0 for c in calls)
    # every distinct option set is measured once
    assert len(hist) == len({tuple(sorted(h[0].items())) for h in hist})


def test_failing_candidates_are_skipped():
    clock, calls = FakeClock(), []

    def cost(kw):
        if kw["fuse_cells"] == 32:
            raise RuntimeError("did not converge")
        return 2.0 if kw["vanka_team_max"] == 0 else 1.0
    P = W.small_case(32, 32, False)
    best, t, hist = autotune.tune(P, precision=0, steps=2, warmup=0,
                                  solver_cls=make_solver(clock, cost, calls), clock=clock)
    assert best["fuse_cells"] != 32 and best["vanka_team_max"] != 0
    assert any(sec is None for _, sec in hist)


def test_table_round_trip(tmp_path):
    P = W.small_case(48, 64, True)
    path = str(tmp_path / "tuned.json")
    key = autotune.key_of(P, 1, 1, 0, "GB300")
    autotune.save_entry(path, key, {"fuse_cells32": 2048, "vanka_team_max32": 0}, 0.0125)
    autotune.save_entry(path, autotune.key_of(P, 0, 0, 0, "GB300"), {"fuse_cells": 32}, 0.03)
    table = autotune.load_table(path)
    assert autotune.lookup(table, P, 1, 1, 0, "GB300") == {"fuse_cells32": 2048,
                                                           "vanka_team_max32": 0}
    assert table[key]["ms_per_step"] == pytest.approx(12.5)
    assert autotune.lookup(table, P, 1, 0, 0, "GB300") == {}
    assert autotune.lookup(table, P, 1, 1, 0, "other GPU") == {}


def test_every_knob_has_the_library_default_first():
    defaults = {"vanka_team_max": 8192, "ch_team_max": 4096, "fuse_cells": 128,
                "vanka_team_max32": 65536, "ch_team_max32": 0, "fuse_cells32": 512,
                "nu1": 2, "nu2": 2, "nu_coarse": 4, "vanka_team8_max": 0, "vanka_pair_max": 0, "vanka_split": 0,
                "coarse_smem": 1,
                "wave_cells32": 0,
                "wave_rows": 8, "skew_cells32": 0, "skew_rows": 32, "nu1_fine": -1, "nu2_fine": -1}
    for k, v in defaults.items():
        assert autotune.CANDIDATES[k][0] == v
    for p, knobs in autotune.KNOBS.items():
        assert all(k in autotune.CANDIDATES for k in knobs)


def test_slow_candidates_are_cut_off_by_the_step_time_limit():
    """After the first measurement every trial carries step_time_limit =
    20 x the best time per step; a candidate slower than that fails its step
    (as qnsch_step's QNSCH_ETIMEOUT would) and is skipped."""
    clock, calls = FakeClock(), []

    def cost(kw):
        c = 100.0 if kw["fuse_cells"] == 4096 else 1.0
        lim = kw.get("step_time_limit", 0.0)
        if lim and c > lim:
            raise RuntimeError("QNSCH_ETIMEOUT")
        return c
    P = W.small_case(32, 32, False)
    best, t, hist = autotune.tune(P, precision=0, steps=2, warmup=0,
                                  solver_cls=make_solver(clock, cost, calls), clock=clock)
    assert "step_time_limit" not in calls[0] and "step_time_limit" not in best
    assert all(c["step_time_limit"] == pytest.approx(20.0) for c in calls[1:])
    assert best["fuse_cells"] != 4096 and t == pytest.approx(1.0)
    assert any(h[0]["fuse_cells"] == 4096 and h[1] is None for h in hist)
