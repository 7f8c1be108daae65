"""The simulation driver's host logic on CPU with a stand-in solver: one JSON
line per committed step with the step's record, checkpoints every `every`
steps and at the end, and a failing step logged with its status, the last
committed state checkpointed and the error raised."""
import io
import json

import pytest

from paper_1703_06606_gb300 import qnsch, run


class FakeSolver:
    def __init__(self, fail_at=None):
        self.fail_at, self.steps, self.saved = fail_at, 0, []

    def step(self, dt):
        if self.fail_at is not None and self.steps + 1 == self.fail_at:
            raise qnsch.QnschError("qnsch_step", -4)
        self.steps += 1
        return 7, 5e-10

    def mass(self):
        return 1.5, 0.25

    def energy(self):
        return 2.0 - 0.01 * self.steps, 0.01

    def save_checkpoint(self, path, t=0.0, n=0):
        self.saved.append((path, round(t, 12), n, self.steps))


def _ticks():
    x = [0.0]

    def clock():
        x[0] += 0.002
        return x[0]
    return clock


def test_log_and_checkpoints():
    s, log = FakeSolver(), io.StringIO()
    t, n = run.simulate(s, 0.1, 5, t=1.0, n=10, log=log, checkpoint="ck.npz", every=2,
                        clock=_ticks())
    assert (round(t, 12), n) == (1.5, 15)
    recs = [json.loads(x) for x in log.getvalue().splitlines()]
    assert [r["step"] for r in recs] == [11, 12, 13, 14, 15]
    r = recs[0]
    assert r["vcycles"] == 7 and r["residual"] == 5e-10 and r["status"] == 0
    assert (r["mass_rho"], r["mass_rhoc"]) == (1.5, 0.25) and r["energy"] == pytest.approx(1.99)
    assert r["wall_ms"] == pytest.approx(2.0)
    assert s.saved == [("ck.npz", 1.2, 12, 2), ("ck.npz", 1.4, 14, 4), ("ck.npz", 1.5, 15, 5)]


def test_failure_is_logged_and_checkpointed():
    s, log = FakeSolver(fail_at=3), io.StringIO()
    with pytest.raises(qnsch.QnschError):
        run.simulate(s, 0.5, 5, log=log, checkpoint="ck.npz", clock=_ticks())
    recs = [json.loads(x) for x in log.getvalue().splitlines()]
    assert [(r["step"], r["status"]) for r in recs] == [(1, 0), (2, 0), (3, -4)]
    assert s.saved == [("ck.npz", 1.0, 2, 2)]


class CliSolver(FakeSolver):
    """Stand-in for qnsch.Solver in run.main: records its construction."""
    made = []

    def __init__(self, **kw):
        super().__init__()
        self.kw = kw
        CliSolver.made.append(self)

    def set_fields(self, f):
        self.fields = f

    def save_checkpoint(self, path, t=0.0, n=0):
        with open(path, "w") as f:
            json.dump({"t": t, "n": n}, f)

    @classmethod
    def from_checkpoint(cls, path, stream=None, **over):
        with open(path) as f:
            d = json.load(f)
        s = cls(resumed=True, **over)
        return s, d["t"], d["n"]


def test_cli_wiring(tmp_path, monkeypatch, capsys):
    from paper_1703_06606_gb300 import workloads as W
    monkeypatch.setattr(run.qnsch, "Solver", CliSolver)
    CliSolver.made.clear()
    log, ck = str(tmp_path / "s.jsonl"), str(tmp_path / "s.ck")
    run.main(["--workload", "small", "--steps", "3", "--tol", "1e-8", "--log", log,
              "--checkpoint", ck, "--every", "2"])
    s = CliSolver.made[-1]
    assert s.kw["tol"] == 1e-8 and s.kw["m1"] == 32 and "c" in s.fields
    assert len(open(log).read().splitlines()) == 3
    assert json.loads(capsys.readouterr().out)["steps"] == 3
    run.main(["--resume", ck, "--steps", "2", "--coupled", "1", "--log", log,
              "--step-time-limit", "2.5", "--diverge-cycles", "3"])
    s = CliSolver.made[-1]
    assert s.kw == {"resumed": True, "coupled": 1, "step_time_limit": 2.5, "diverge_cycles": 3}
    assert [json.loads(x)["step"] for x in open(log).read().splitlines()] == [1, 2, 3, 4, 5]
    cfg = tmp_path / "p.json"
    P = W.small_case(24, 16, False)
    cfg.write_text(P.to_json())
    run.main(["--config", str(cfg), "--steps", "1"])
    s = CliSolver.made[-1]
    assert (s.kw["m1"], s.kw["m2"], s.kw["periodic_x"], s.kw["tol"]) == (24, 16, False, P.tol)
