"""Exact identities of the oracle's building blocks, on random inputs.

Secants (Sec. 4.1): F(a) - F(b) = g(a,b)(a - b) for the double well
F(c) = c^2 (c-1)^2 / 4, with g(a,a) = F'(a) = a(a-1)(a-1/2); rho(a) - rho(b) =
r(a,b)(a - b) for rho(c) = rho1 rho2 / ((rho2 - rho1) c + rho1) and
r = -alpha rho(a) rho(b); rho(1) = rho1, rho(0) = rho2; dg/da against central
differences.

Summation by parts (App. A): the CH operator L phi = grad_d.(A m^n grad_D phi)
is read off the residual of (pm-num-phase) with c = c^n, u = v = p = 0 and
mu = phi, where the time, advection and pressure terms vanish and
r_c = (1/Pe) L phi.  With Neumann walls or periodic x, for random positive
mobility and random phi, psi: <psi, L phi> = <phi, L psi> (self-adjoint),
<phi, L phi> < 0 for non-constant phi and sum L phi = 0 (the fluxes cancel),
L 1 = 0.  A wrong ghost value, a one-sided average or a dropped face breaks
one of them.

Adjointness and definiteness of the momentum and mass rows: the discrete
pressure gradient is minus the adjoint of the discrete divergence, and the
momentum rows at rest are symmetric positive definite.

Grid transfers (reading R8): the residual restriction is the area-weighted
adjoint of the correction prolongation, for cells and both edge families,
and R P = I on cells."""
import numpy as np
import pytest

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W


def _solver(m1=12, m2=10, px=False, rho1=1.0, rho2=3.0):
    return RefSolver(m1, m2, periodic_x=px, rho1=rho1, rho2=rho2, eta1=1.0, eta2=2.0, Re=50.0,
                     We=5.0, Pe=20.0, Cn=0.05, Fr=0.8)


@pytest.mark.parametrize("rho1,rho2", [(1.0, 3.0), (1000.0, 1.0), (0.1, 1.0)])
def test_secant_identities(rho1, rho2):
    s = _solver(rho1=rho1, rho2=rho2)
    rng = np.random.default_rng(11)
    for a, b in rng.uniform(-0.5, 1.5, size=(200, 2)):
        x = s.secants(a, b)
        scale = 1.0 + abs(x["Fa"]) + abs(x["Fb"])
        assert abs((x["Fa"] - x["Fb"]) - x["g"] * (a - b)) <= 4e-16 * scale * 8
        rs = max(abs(x["rho_a"]), abs(x["rho_b"]))
        assert abs((x["rho_a"] - x["rho_b"]) - x["r"] * (a - b)) <= 1e-14 * rs * (1 + abs(a - b))
        e = 1e-6
        fd = (s.secants(a + e, b)["g"] - s.secants(a - e, b)["g"]) / (2 * e)
        assert abs(fd - x["g_a"]) <= 1e-8 * (1 + abs(fd))
        assert abs(s.secants(a, a)["g"] - a * (a - 1) * (a - 0.5)) <= 1e-15 * (1 + abs(a) ** 3)
    one, zero = s.secants(1.0, 0.0)["rho_a"], s.secants(1.0, 0.0)["rho_b"]
    assert abs(one - rho1) <= 1e-14 * rho1 and abs(zero - rho2) <= 1e-14 * rho2


def _begin(s, cn, dt=1e-2):
    """Freeze c^n (and u^n = v^n = 0) for the operators of the step."""
    s.set_fields(dict(s.zeros(), c=cn))
    s.begin_step(dt)


def _L(s, cn, phi):
    """(1/Pe) grad_d.(A m(c^n) grad_D phi), up to the residual's sign, from the
    residual of N_c at the iterate c = c^n, u = v = p = 0, mu = phi."""
    s.set_iterate(dict(s.zeros(), c=cn, mu=phi))
    r, _ = s.residual()
    return r["c"]


@pytest.mark.parametrize("px", [False, True])
def test_ch_operator_is_self_adjoint_and_conservative(px):
    m1, m2 = 12, 10
    s = _solver(m1, m2, px)
    rng = np.random.default_rng(5 + int(px))
    cn = rng.uniform(0.05, 0.95, size=(m2, m1))
    phi, psi = rng.standard_normal((2, m2, m1))
    _begin(s, cn)
    Lphi, Lpsi = _L(s, cn, phi), _L(s, cn, psi)
    a, b = float(np.sum(psi * Lphi)), float(np.sum(phi * Lpsi))
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b)), (a, b)
    q1, q2 = float(np.sum(phi * Lphi)), float(np.sum(psi * Lpsi))
    assert q1 != 0.0 and np.sign(q1) == np.sign(q2)
    assert abs(np.sum(Lphi)) <= 1e-12 * np.sum(np.abs(Lphi))
    L1 = _L(s, cn, np.ones((m2, m1)))
    assert np.max(np.abs(L1)) <= 1e-12
    # the sign is that of -(1/Pe)<grad phi, A m grad phi> on either side of the
    # residual convention; both quadratic forms agree, and a constant is in
    # the kernel, so the operator is semi-definite on this grid


@pytest.mark.parametrize("px", [False, True])
def test_pressure_gradient_is_minus_adjoint_of_divergence(px):
    """h^2 sum_cells p (d.u) = -h^2 sum_edges (D p).u for u vanishing on walls
    (App. A): the (1/M) D p of (pm-num-mx) and the d.u of (pm-num-mass), read
    off the residuals.  With u^n = v^n = 0, c = c^n, mu = 0 and no gravity,
    a state with only p nonzero gives r_u = -(1/M) D_x p, r_v = -(1/M) D_y p,
    and a state with only u, v nonzero gives r_p = -(d_x u + d_y v)."""
    m1, m2 = 12, 10
    s = RefSolver(m1, m2, periodic_x=px, rho1=1.0, rho2=3.0, eta1=1.0, eta2=2.0, Re=50.0,
                  We=5.0, Pe=20.0, Cn=0.05, Fr=float("inf"))
    M = s.params()["M"]
    rng = np.random.default_rng(9 + int(px))
    cn = rng.uniform(0.05, 0.95, size=(m2, m1))
    _begin(s, cn)
    z = s.zeros()
    p = rng.standard_normal((m2, m1))
    u, v = rng.standard_normal(z["u"].shape), rng.standard_normal(z["v"].shape)
    v[0, :] = v[-1, :] = 0.0  # walls in y
    if px:
        u[:, 0] = u[:, -1]  # one unknown
    else:
        u[:, 0] = u[:, -1] = 0.0  # walls in x
    s.set_iterate(dict(z, c=cn, p=p))
    rp_state, _ = s.residual()
    s.set_iterate(dict(z, c=cn, u=u, v=v))
    ru_state, _ = s.residual()
    cols = slice(1, m1 + 1)  # periodic: columns 0 and m1 are one edge
    lhs = float(np.sum(p * -ru_state["p"]))                    # sum p (d.u)
    Du = -M * rp_state["u"][:, cols]                          # D_x p on the x-edges
    Dv = -M * rp_state["v"]                                   # D_y p on the y-edges
    rhs = -(float(np.sum(Du * u[:, cols])) + float(np.sum(Dv * v)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)), (lhs, rhs)


def _edge_parts(r, m1, px):
    """The unknowns of the x- and y-edge arrays (periodic x: columns 0 and m1
    are one edge; walls: their entries are not unknowns)."""
    if px:
        return r["u"][:, 1:m1 + 1], r["v"][1:-1, :]
    return r["u"][:, 1:m1], r["v"][1:-1, :]


@pytest.mark.parametrize("px", [False, True])
def test_momentum_operator_at_rest_is_symmetric_positive(px):
    """With u^n = v^n = 0, c = c^n, mu = p = 0 and no gravity, the momentum rows
    of (pm-num-mx) reduce to A rho^n u/dt (diagonal) plus the viscous terms,
    (e1e1) included: a symmetric, positive definite operator on the interior
    edges (its quadratic form is the kinetic-energy term plus the viscous
    dissipation of Thm. 6.2).  Read off the residuals, r = -N."""
    m1, m2 = 12, 10
    s = RefSolver(m1, m2, periodic_x=px, rho1=1.0, rho2=3.0, eta1=1.0, eta2=20.0, Re=0.5,
                  We=5.0, Pe=20.0, Cn=0.05, Fr=float("inf"))
    rng = np.random.default_rng(13 + int(px))
    cn = rng.uniform(0.05, 0.95, size=(m2, m1))
    _begin(s, cn, dt=1.0)
    z = s.zeros()

    def field(seed):
        g = np.random.default_rng(seed)
        u, v = g.standard_normal(z["u"].shape), g.standard_normal(z["v"].shape)
        v[0, :] = v[-1, :] = 0.0
        if px:
            u[:, 0] = u[:, -1]
        else:
            u[:, 0] = u[:, -1] = 0.0
        return u, v

    def N(u, v):
        s.set_iterate(dict(z, c=cn, u=u, v=v))
        r, _ = s.residual()
        nu, nv = _edge_parts(r, m1, px)
        return -nu, -nv

    (u1, v1), (u2, v2) = field(1), field(2)
    a_u, a_v = N(u1, v1)
    b_u, b_v = N(u2, v2)
    e1u, e1v = _edge_parts({"u": u1, "v": v1}, m1, px)
    e2u, e2v = _edge_parts({"u": u2, "v": v2}, m1, px)
    x = float(np.sum(e2u * a_u) + np.sum(e2v * a_v))
    y = float(np.sum(e1u * b_u) + np.sum(e1v * b_v))
    # the cross terms cancel between entries of order mu/(Re h^2): rounding is
    # relative to the sum of the products' magnitudes
    mag = float(np.sum(np.abs(e2u * a_u)) + np.sum(np.abs(e2v * a_v)))
    assert abs(x - y) <= 1e-13 * mag, (x, y, mag)
    q = float(np.sum(e1u * a_u) + np.sum(e1v * a_v))
    kin = float(np.sum(e1u ** 2) + np.sum(e1v ** 2))
    assert q > 0.0 and q > 0.1 * kin  # the time term alone gives about rho * kin


def _shapes(m1, m2):
    return {0: (m2, m1), 1: (m2, m1 + 1), 2: (m2 + 1, m1)}


def _unknowns(fam, m1, m2, px):
    """Mask of the unknowns of a family in its host layout (walls excluded;
    with periodic x, x-edge 0 is edge m1)."""
    mask = np.ones(_shapes(m1, m2)[fam], dtype=bool)
    if fam == 1:
        mask[:, 0] = False
        if not px:
            mask[:, m1] = False
    if fam == 2:
        mask[0, :] = mask[m2, :] = False
    return mask


@pytest.mark.parametrize("px", [False, True])
def test_transfers_restriction_is_the_scaled_adjoint_of_prolongation(px):
    """Reading R8: with area weights h^2 on the fine and (2h)^2 on the coarse
    level, <R r, e>_H = <r, P e>_h for cells (average / piecewise constant) and
    for both edge families (full weighting / linear in the normal direction),
    over the unknowns; and R P = I on cells."""
    m1, m2 = 16, 12
    s = _solver(m1, m2, px)
    rng = np.random.default_rng(21 + int(px))
    M1, M2 = m1 // 2, m2 // 2
    for fam in (0, 1, 2):
        fine_mask = _unknowns(fam, m1, m2, px)
        coarse_mask = _unknowns(fam, M1, M2, px)
        r = rng.standard_normal(_shapes(m1, m2)[fam]) * fine_mask
        e = rng.standard_normal(_shapes(M1, M2)[fam]) * coarse_mask
        if fam == 1 and px:  # edge 0 is edge m1: the same unknown
            r[:, 0] = r[:, m1]
            e[:, 0] = e[:, M1]
        Rr = s.transfer(0, fam, r, _shapes(M1, M2)[fam])
        Pe = s.transfer(0, 3 + fam, e, _shapes(m1, m2)[fam])
        lhs = 4.0 * float(np.sum((Rr * e)[coarse_mask]))
        rhs = float(np.sum((r * Pe)[fine_mask]))
        assert abs(lhs - rhs) <= 1e-13 * (np.sum(np.abs(r)) * np.max(np.abs(e))), (fam, lhs, rhs)
    ec = rng.standard_normal((M2, M1))
    back = s.transfer(0, 0, s.transfer(0, 3, ec, (m2, m1)), (M2, M1))
    assert np.array_equal(back, ec)


@pytest.mark.parametrize("px", [False, True])
def test_state_restriction_of_edges(px):
    """Reading R8: a coarse edge's state is the mean of the two fine edges that
    lie on it.  So a fine field that is antisymmetric across each such pair
    restricts to zero, a constant stays constant, and restricting a
    prolongated coarse field returns it."""
    m1, m2 = 16, 12
    s = _solver(m1, m2, px)
    M1, M2 = m1 // 2, m2 // 2
    rng = np.random.default_rng(31 + int(px))
    # x-edges: fine rows 2J-1 and 2J lie on coarse row J
    a = rng.standard_normal((M2, m1 + 1))
    u = np.repeat(a, 2, axis=0) * np.tile([1.0, -1.0], M2)[:, None]
    assert np.max(np.abs(s.transfer(0, 6, u, (M2, M1 + 1)))) == 0.0
    ones = s.transfer(0, 6, np.full((m2, m1 + 1), 1.5), (M2, M1 + 1))
    assert np.all(ones == 1.5)
    # y-edges: fine columns 2I-1 and 2I lie on coarse column I
    b = rng.standard_normal((m2 + 1, M1))
    v = np.repeat(b, 2, axis=1) * np.tile([1.0, -1.0], M1)[None, :]
    assert np.max(np.abs(s.transfer(0, 7, v, (M2 + 1, M1)))) == 0.0
    for fam, op, shape_c, shape_f in ((1, 6, (M2, M1 + 1), (m2, m1 + 1)),
                                      (2, 7, (M2 + 1, M1), (m2 + 1, m1))):
        e = rng.standard_normal(shape_c) * _unknowns(fam, M1, M2, px)
        if fam == 1 and px:
            e[:, 0] = e[:, M1]
        back = s.transfer(0, op, s.transfer(0, 3 + fam, e, shape_f), shape_c)
        mask = _unknowns(fam, M1, M2, px)
        assert np.allclose(back[mask], e[mask], rtol=0, atol=1e-15)
