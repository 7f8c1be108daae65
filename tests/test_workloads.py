"""The synthetic inputs: each workload has the grid, boundaries, parameters and
initial profile of the example of Sec. 8 it stands in for, the batch and the
request stream draw from the stated distributions, and every generator is
deterministic for its seed."""
import math

import numpy as np

from paper_1703_06606_gb300 import serve
from paper_1703_06606_gb300 import workloads as W


def _at(P, c, x, y):
    """c at the cell containing (x, y)."""
    return c[int(y / P.h), int(x / P.h)]


def test_rising_drop():
    P = W.rising_drop_256x512()
    assert (P.m1, P.m2, P.periodic_x, P.m2 * P.h) == (256, 512, False, 2.0)
    assert (P.rho1, P.rho2, P.eta1, P.eta2) == (0.1, 1.0, 0.1, 1.0)
    assert (P.Re, P.We, P.Fr, P.Cn, P.dt, P.tol) == (35.0, 10.0, 1.0, 0.01, 2e-4, 1e-9)
    f = P.fields()
    c = f["c"]
    assert _at(P, c, 0.5, 0.5) > 0.999 and _at(P, c, 0.05, 1.9) < 1e-3
    # the c = 1/2 level set at radius 0.25 about (0.5, 0.5)
    row = c[int(0.5 / P.h)]
    x = (np.arange(P.m1) + 0.5) * P.h
    i = np.argmin(np.abs(row[x > 0.5] - 0.5))
    assert abs(x[x > 0.5][i] - 0.75) <= P.h
    assert all(np.all(f[k] == 0.0) for k in ("mu", "p", "u", "v"))


def test_capillary_and_rayleigh_taylor():
    P = W.capillary_64()
    assert (P.m1, P.m2, P.periodic_x, math.isinf(P.Fr), P.tol) == (64, 64, True, True, 1e-10)
    c = P.fields()["c"]
    height = P.h * c.sum(axis=0)  # c = 1 below the interface
    x = (np.arange(P.m1) + 0.5) * P.h
    assert np.max(np.abs(height - (0.5 + 0.01 * np.cos(2 * math.pi * x)))) < 1e-3
    R = W.rayleigh_taylor_1024x4096()
    assert (R.m1, R.m2, R.periodic_x, R.m2 * R.h, R.Cn) == (1024, 4096, True, 4.0, 0.005)
    assert (R.rho1, R.rho2, R.Re, R.We) == (1.0, 3.0, 3000.0, 200.0)  # light (c = 1) below


def test_batch_drops():
    probs = W.batch_drops(64)
    assert len(probs) == 64
    grids = {(64, 64), (128, 128), (256, 512), (512, 512)}
    for P in probs:
        assert (P.m1, P.m2) in grids and not P.periodic_x
        assert 2.0 <= P.rho2 / P.rho1 <= 100.0 and 1.0 <= P.eta2 / P.eta1 <= 50.0
        assert P.Cn == 2.5 / P.m1 and abs(P.Pe * P.Cn - 1.0) < 1e-12
        assert 0.15 <= P.init_args["R"] <= 0.3
    assert len({(P.m1, P.m2) for P in probs}) == 4
    again = W.batch_drops(64)
    assert [(P.m1, P.rho1, P.init_args["R"]) for P in probs] == \
           [(P.m1, P.rho1, P.init_args["R"]) for P in again]


def test_request_stream():
    reqs = serve.poisson_requests(400, rate=50.0, n_min=128, n_max=1024, steps=50, dt=1e-4)
    t = [r.arrival for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    assert 0.8 * 400 / 50.0 < t[-1] < 1.2 * 400 / 50.0  # mean inter-arrival 1/50 s
    Ns = [r.problem.m1 for r in reqs]
    assert all(N % 64 == 0 and 128 <= N <= 1024 and r.problem.m2 == N
               for N, r in zip(Ns, reqs))
    caps = sum(1 for r in reqs if r.problem.init == "capillary")
    assert 0.4 * 400 < caps < 0.6 * 400
    # log-uniform: as many sides below the geometric mean of the range as above
    below = sum(1 for N in Ns if N < math.sqrt(128 * 1024))
    assert 0.35 * 400 < below < 0.65 * 400


def test_generators_are_deterministic():
    for make in (W.rising_drop_256x512, W.capillary_64, lambda: W.small_case(24, 16, False)):
        a, b = make().fields(), make().fields()
        assert all(np.array_equal(a[k], b[k]) for k in a)
    r1 = W.random_state(16, 12, True, seed=4)
    r2 = W.random_state(16, 12, True, seed=4)
    assert all(np.array_equal(r1[k], r2[k]) for k in r1)
