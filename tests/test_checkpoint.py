"""Checkpoint files on CPU: a save/load round trip keeps the fields bit for
bit, the parameters (an infinite Froude number included), the options, t and
n; wrong shapes, missing parameters and an unknown format are refused; a
failed write leaves no partial file in place."""
import json

import numpy as np
import pytest

from paper_1703_06606_gb300 import checkpoint as C
from paper_1703_06606_gb300 import workloads as W


def _state(m1=24, m2=16, px=True):
    P = W.small_case(m1, m2, px)
    params = dict(P.create_kwargs())
    rng = np.random.default_rng(3)
    fields = {k: rng.standard_normal(s) for k, s in C.field_shapes(m1, m2).items()}
    opts = {"scheme": 0.0, "precision": 1.0, "coupled": 1.0, "tol": 1e-9, "fuse_cells32": 2048.0}
    return fields, params, opts


def test_round_trip(tmp_path):
    fields, params, opts = _state()
    params["Fr"] = float("inf")
    path = str(tmp_path / "a.npz")
    C.save(path, fields, params, opts, t=0.125, n=17)
    f2, p2, o2, t, n = C.load(path)
    for k in C.FIELDS:
        assert f2[k].dtype == np.float64 and np.array_equal(f2[k], fields[k])
    assert p2 == params and o2 == opts and t == 0.125 and n == 17
    assert list(o2) == [k for k in C.OPTIONS if k in opts]  # restore order


def test_refusals(tmp_path):
    fields, params, opts = _state()
    bad = dict(fields, u=fields["u"][:, :-1])
    with pytest.raises(ValueError):
        C.save(str(tmp_path / "b.npz"), bad, params, opts)
    with pytest.raises(ValueError):
        C.save(str(tmp_path / "b.npz"), fields, {k: v for k, v in params.items() if k != "Re"},
               opts)
    assert not list(tmp_path.iterdir())
    path = str(tmp_path / "c.npz")
    meta = {"format": 99, "params": params, "options": {}, "t": 0.0, "n": 0}
    np.savez(path, meta=np.array(json.dumps(meta)), **fields)
    with pytest.raises(ValueError):
        C.load(path)


def test_problem_json_round_trip():
    for P in (W.rising_drop_256x512(), W.capillary_64(), W.rayleigh_taylor_1024x4096(),
              W.small_case(24, 16, True)):
        Q = W.Problem.from_json(P.to_json())
        assert Q == P
        for k, a in P.fields().items():
            assert np.array_equal(Q.fields()[k], a)
    with pytest.raises(ValueError):
        W.Problem.from_json('{"name": "x", "grid": 3}')


def test_hand_written_problem_json():
    """A problem written by hand: init and init_args may be left out (a flat
    interface at mid-height, the capillary profile), Infinity is no gravity."""
    text = ('{"name": "mine", "m1": 48, "m2": 32, "Lx": 1.5, "periodic_x": true, "levels": 0,'
            ' "rho1": 1.0, "rho2": 2.0, "eta1": 1.0, "eta2": 1.0, "Re": 100.0, "We": 10.0,'
            ' "Pe": 50.0, "Cn": 0.02, "Fr": Infinity, "dt": 0.001, "steps": 5, "tol": 1e-9}')
    P = W.Problem.from_json(text)
    assert P.init == "capillary" and P.init_args == {} and np.isinf(P.Fr)
    assert P.h == 1.5 / 48 and P.create_kwargs()["periodic_x"] is True
    c = P.fields()["c"]
    assert c.shape == (32, 48) and c[0, 0] > 0.99 and c[-1, 0] < 0.01
