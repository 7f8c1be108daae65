"""Seeded synthetic workloads: grids, physical parameters and initial fields.

This module holds no arithmetic of the method itself (no discrete operator, no
solver step); it only builds inputs.  Both the CUDA path's tests and benchmarks
and the oracle's tests use it.

Workloads follow the examples of Sec. 8 of Guo, Lin, Lowengrub & Wise
(arXiv:1703.06606): a capillary wave (Sec. 8.1), a rising droplet (Sec. 8.2) and a
Rayleigh-Taylor interface (Sec. 8.3), with diffuse-interface initial profiles
c = 1/2 (1 - tanh(d / (2 sqrt(2) Cn))), where d is the signed distance-like
coordinate of each example (2 sqrt(2) Cn is the equilibrium width of the profile
for F(c) = c^2 (c-1)^2 / 4).

Array layouts (numpy, C order, no ghost cells):
    c, mu, p : (m2, m1); u : (m2, m1 + 1); v : (m2 + 1, m1)
"""
from __future__ import annotations

import dataclasses
import json
import math

import numpy as np

SEED = 1703066


@dataclasses.dataclass
class Problem:
    name: str
    m1: int
    m2: int
    Lx: float
    periodic_x: bool
    levels: int  # 0 = the deepest hierarchy the grid allows
    rho1: float
    rho2: float
    eta1: float
    eta2: float
    Re: float
    We: float
    Pe: float
    Cn: float
    Fr: float
    dt: float
    steps: int
    tol: float
    init: str = "capillary"
    init_args: dict = dataclasses.field(default_factory=dict)

    @property
    def h(self):
        return self.Lx / self.m1

    @property
    def cells(self):
        return self.m1 * self.m2

    def create_kwargs(self):
        return dict(m1=self.m1, m2=self.m2, Lx=self.Lx, periodic_x=self.periodic_x,
                    levels=self.levels, rho1=self.rho1, rho2=self.rho2, eta1=self.eta1,
                    eta2=self.eta2, Re=self.Re, We=self.We, Pe=self.Pe, Cn=self.Cn, Fr=self.Fr)

    def fields(self):
        return initial_fields(self)

    def to_json(self):
        """The problem as a JSON object (an infinite Froude number as Infinity)."""
        return json.dumps(dataclasses.asdict(self), sort_keys=True)

    @classmethod
    def from_json(cls, text):
        """A problem from to_json's text, or from a hand-written JSON object
        with the same keys (init and init_args may be left out)."""
        d = json.loads(text)
        names = {f.name for f in dataclasses.fields(cls)}
        unknown = set(d) - names
        if unknown:
            raise ValueError("unknown problem keys: %s" % sorted(unknown))
        return cls(**d)


def cell_centres(m1, m2, h):
    x = (np.arange(1, m1 + 1) - 0.5) * h
    y = (np.arange(1, m2 + 1) - 0.5) * h
    return np.meshgrid(x, y)  # (m2, m1)


def _profile(d, Cn):
    return 0.5 * (1.0 - np.tanh(d / (2.0 * math.sqrt(2.0) * Cn)))


def initial_fields(P: Problem):
    X, Y = cell_centres(P.m1, P.m2, P.h)
    a = P.init_args
    if P.init == "capillary":
        # interface y = y0 + H0 cos(2 pi k x / Lx), k = 1 unless given; c = 1 below
        # (Sec. 8.1 profile)
        y0, H0, kx = a.get("y0", 0.5 * P.m2 * P.h), a.get("H0", 0.01), a.get("k", 1)
        c = _profile(Y - y0 - H0 * np.cos(2.0 * math.pi * kx * X / P.Lx), P.Cn)
    elif P.init == "drop":
        # circular drop (c = 1) of radius R centred at (x0, y0), Sec. 8.2
        x0, y0, R = a.get("x0", 0.5), a.get("y0", 0.5), a.get("R", 0.25)
        c = _profile(np.sqrt((X - x0) ** 2 + (Y - y0) ** 2) - R, P.Cn)
    elif P.init == "rt":
        # light fluid (c = 1) below y = y0 + A cos(2 pi x), Sec. 8.3
        y0, A = a.get("y0", 2.0), a.get("A", 0.1)
        c = _profile(Y - y0 - A * np.cos(2.0 * math.pi * X / P.Lx), P.Cn)
    elif P.init == "cosines":
        # c = cos(2 pi x) + cos(2 pi y), the initial state of the convergence test (Sec. 9)
        c = np.cos(2.0 * math.pi * X) + np.cos(2.0 * math.pi * Y)
    else:
        raise ValueError(P.init)
    z = dict(c=c, mu=np.zeros((P.m2, P.m1)), p=np.zeros((P.m2, P.m1)),
             u=np.zeros((P.m2, P.m1 + 1)), v=np.zeros((P.m2 + 1, P.m1)))
    return z


# ---------------------------------------------------------------------------
# the five workloads of the benchmark suite
# ---------------------------------------------------------------------------

def capillary_64():
    """Capillary wave 64x64 on [0,1]^2, periodic x, walls y, rho 1:1, no gravity."""
    return Problem("capillary_wave_64x64", 64, 64, 1.0, True, 0, 1.0, 1.0, 1.0, 1.0,
                   Re=100.0, We=10.0, Pe=100.0, Cn=0.01, Fr=math.inf, dt=1e-3, steps=10,
                   tol=1e-10, init="capillary", init_args=dict(y0=0.5, H0=0.01))


def rising_drop_256x512():
    """Rising droplet 256x512 on [0,1]x[0,2], walls all round.  The drop (c = 1) is
    the light fluid: rho1 = 0.1, mu1 = 0.1 inside, rho2 = mu2 = 1 outside."""
    return Problem("rising_droplet_256x512", 256, 512, 1.0, False, 0, 0.1, 1.0, 0.1, 1.0,
                   Re=35.0, We=10.0, Pe=100.0, Cn=0.01, Fr=1.0, dt=2e-4, steps=200,
                   tol=1e-9, init="drop", init_args=dict(x0=0.5, y0=0.5, R=0.25))


def rayleigh_taylor_1024x4096():
    """Rayleigh-Taylor, At = 0.5 (rho 1:3), light fluid (c = 1) below y = 2 + 0.1 cos(2 pi x)."""
    return Problem("rayleigh_taylor_1024x4096", 1024, 4096, 1.0, True, 0, 1.0, 3.0, 1.0, 1.0,
                   Re=3000.0, We=200.0, Pe=200.0, Cn=0.005, Fr=1.0, dt=1e-4, steps=100,
                   tol=1e-9, init="rt", init_args=dict(y0=2.0, A=0.1))


def capillary_ratio1000_256():
    """Capillary wave at density ratio 1:1000 (case 2 of Sec. 8.1): 256x256 on
    [0,1]^2, periodic x, equal kinematic viscosities (mu = rho), Re = 100,
    We = 1, Fr = 1, Cn = 0.005, Pe = 1/Cn, dt = 1e-3.  The heavy fluid (c = 1)
    lies below the interface 0.5 + 0.01 cos(2 pi x), a gravity-capillary wave."""
    return Problem("capillary_ratio1000_256", 256, 256, 1.0, True, 0, 1000.0, 1.0, 1000.0, 1.0,
                   Re=100.0, We=1.0, Pe=200.0, Cn=0.005, Fr=1.0, dt=1e-3, steps=20, tol=1e-9,
                   init="capillary", init_args=dict(y0=0.5, H0=0.01))


def droplet_paper_256x512():
    """The droplet with the paper's own parameters (Sec. 8.2): rho and mu ratio
    1:10 (drop c = 1 light), Re = 100, We = 1, Fr = 0.98, Cn = 0.005, Pe = 1/Cn,
    dt = 1e-3, on [0,1]x[0,2], 256x512, periodic x, drop of radius 0.25 at
    (0.5, 0.5)."""
    return Problem("droplet_paper_256x512", 256, 512, 1.0, True, 0, 0.1, 1.0, 0.1, 1.0,
                   Re=100.0, We=1.0, Pe=200.0, Cn=0.005, Fr=0.98, dt=1e-3, steps=20, tol=1e-9,
                   init="drop", init_args=dict(x0=0.5, y0=0.5, R=0.25))


def convergence_test(m):
    """The self-convergence test of Sec. 9 on level m (m = 16, 32, ..., 256):
    [0,1]^2 with walls, c = cos(2 pi x) + cos(2 pi y), everything else zero,
    dt = 16 h^2 (1/16 at m = 16, 1/4096 at m = 256).  The paper leaves the
    physical parameters open; c reaches -2 and 2, where rho(c) would be
    singular for rho1 != rho2, so rho1 = rho2 = 1, mu1 = mu2 = 1, Re = 100,
    We = 10, Cn = 0.05, Pe = 1/Cn, no gravity."""
    return Problem("convergence_%d" % m, m, m, 1.0, False, 0, 1.0, 1.0, 1.0, 1.0,
                   Re=100.0, We=10.0, Pe=20.0, Cn=0.05, Fr=math.inf, dt=16.0 / (m * m),
                   steps=m * m // 256, tol=1e-11, init="cosines")


def batch_drops(n=64, seed=SEED):
    """n independent rising-drop instances with seeded grids and parameters."""
    rng = np.random.default_rng(seed)
    grids = [(64, 64), (128, 128), (256, 512), (512, 512)]
    out = []
    for k in range(n):
        m1, m2 = grids[rng.integers(0, len(grids))]
        R = rng.uniform(0.15, 0.3)
        ratio_rho = rng.uniform(2.0, 100.0)
        ratio_mu = rng.uniform(1.0, 50.0)
        Cn = 2.5 / m1
        Ly = m2 / m1
        out.append(Problem("drop_%d" % k, m1, m2, 1.0, False, 0, 1.0 / ratio_rho, 1.0,
                           1.0 / ratio_mu, 1.0, Re=35.0, We=10.0, Pe=1.0 / Cn, Cn=Cn, Fr=1.0,
                           dt=2e-4, steps=20, tol=1e-9, init="drop",
                           init_args=dict(x0=0.5, y0=min(0.5, 0.5 * Ly), R=R)))
    return out


def small_case(m1=32, m2=32, periodic_x=True, rho_ratio=3.0, seed=SEED):
    """A small capillary-type case that exercises every term (rho1 != rho2,
    mu1 != mu2, gravity on)."""
    return Problem("small_%dx%d" % (m1, m2), m1, m2, 1.0, periodic_x, 0, 1.0, rho_ratio, 1.0,
                   2.0, Re=100.0, We=10.0, Pe=1.0 / 0.04, Cn=0.04, Fr=1.0, dt=1e-3, steps=2,
                   tol=1e-10, init="capillary",
                   init_args=dict(y0=0.5 * m2 / m1, H0=0.05))


def random_state(m1, m2, periodic_x, seed=SEED, scale=None):
    """Seeded random fields (c in (0.05, 0.95)) for operator and identity tests."""
    rng = np.random.default_rng(seed)
    s = dict(c=0.5, mu=0.3, p=0.2, u=0.1, v=0.1)
    if scale:
        s.update(scale)
    f = dict(c=0.5 + 0.45 * (2 * rng.random((m2, m1)) - 1) * (s["c"] / 0.5),
             mu=s["mu"] * rng.standard_normal((m2, m1)),
             p=s["p"] * rng.standard_normal((m2, m1)),
             u=s["u"] * rng.standard_normal((m2, m1 + 1)),
             v=s["v"] * rng.standard_normal((m2 + 1, m1)))
    f["c"] = np.clip(f["c"], 0.05, 0.95)
    f["v"][0, :] = 0.0
    f["v"][-1, :] = 0.0
    if periodic_x:
        f["u"][:, 0] = f["u"][:, -1]
    else:
        f["u"][:, 0] = 0.0
        f["u"][:, -1] = 0.0
    return f
