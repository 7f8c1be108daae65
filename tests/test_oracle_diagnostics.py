"""Pins of the oracle's diagnostics of the experiments of Sec. 8 (rise velocity,
centroid, discrete divergence, capillary mode amplitude, interface tips),
each against a closed form computed here from the definition, on states
built so that the discrete value is known exactly."""
import math

import numpy as np
import pytest

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W


def _linear_interface(s, ytilde, slope_cells=4.0):
    """c = clip(1/2 - (y - ytilde(x)) / (slope_cells h), 0, 1): piecewise linear
    across the interface, so the c = 1/2 crossing found by linear
    interpolation between cell centres is exactly ytilde."""
    h = 1.0 / s.m1
    y = (np.arange(1, s.m2 + 1) - 0.5) * h
    return np.clip(0.5 - (y[:, None] - ytilde[None, :]) / (slope_cells * h), 0.0, 1.0)


def test_divergence_of_trigonometric_and_quadratic_fields():
    """u_{i+1/2} = sin(2 pi x_{i+1/2}) (periodic) and v_{j+1/2} = y(Ly - y)
    (zero on the walls): d_x u = 2 sin(pi h)/h cos(2 pi x_i) and d_y v =
    Ly - 2 y_j, exactly for the central differences."""
    m1, m2 = 32, 16
    h = 1.0 / m1
    Ly = m2 * h
    s = RefSolver(m1, m2, periodic_x=True)
    f = s.zeros()
    f["c"][:] = 0.5
    xe = np.arange(m1 + 1) * h
    f["u"][:] = np.sin(2 * math.pi * xe)[None, :]
    ye = np.arange(m2 + 1) * h
    f["v"][:] = (ye * (Ly - ye))[:, None]
    s.set_fields(f)
    xc = (np.arange(1, m1 + 1) - 0.5) * h
    yc = (np.arange(1, m2 + 1) - 0.5) * h
    want = 2 * math.sin(math.pi * h) / h * np.cos(2 * math.pi * xc)[None, :] + (Ly - 2 * yc)[:, None]
    got = s.divergence()
    assert got.shape == (m2, m1)
    assert np.max(np.abs(got - want)) <= 1e-12
    d = s.diagnostics()
    assert abs(d["div_max"] - np.max(np.abs(want))) <= 1e-12
    assert abs(d["div_expansion"] - np.max(want)) <= 1e-12
    assert abs(d["div_compression"] - np.max(-want)) <= 1e-12
    assert abs(d["div_l2"] - math.sqrt(h * h * np.sum(want ** 2))) <= 1e-12


def test_rise_velocity_and_centroid_of_a_translating_block():
    """c = 1 on a block of cells away from the walls, v = V on every interior
    ns edge: V_c = V and the centroid is the block's centre, exactly."""
    m1, m2 = 32, 64
    h = 1.0 / m1
    s = RefSolver(m1, m2, periodic_x=False)
    f = s.zeros()
    f["c"][20:44, 8:24] = 1.0  # rows j = 21..44, columns i = 9..24
    V = 0.3
    f["v"][1:m2, :] = V
    s.set_fields(f)
    d = s.diagnostics()
    assert abs(d["Vc"] - V) <= 1e-13
    assert abs(d["yc"] - 32 * h) <= 1e-14
    # walls: v = 0 on the boundary rows, u = 0 -> divergence only at the first/last rows
    div = s.divergence()
    assert np.all(div[1:m2 - 1, :] == 0.0)
    assert np.allclose(div[0, :], V / h) and np.allclose(div[m2 - 1, :], -V / h)


@pytest.mark.parametrize("a,y0", [(0.01, 0.5), (-0.03, 0.37)])
def test_capillary_mode_amplitude_of_exact_column_heights(a, y0):
    """Column heights h sum_j c_ij = y0 + a cos(2 pi x_i) exactly (c is the cell
    fraction below the interface): a1 = a by discrete orthogonality."""
    m1, m2 = 48, 48
    h = 1.0 / m1
    s = RefSolver(m1, m2, periodic_x=True)
    x = (np.arange(1, m1 + 1) - 0.5) * h
    eta = y0 + a * np.cos(2 * math.pi * x)
    ybot = (np.arange(1, m2 + 1) - 1) * h
    f = s.zeros()
    f["c"][:] = np.clip((eta[None, :] - ybot[:, None]) / h, 0.0, 1.0)
    s.set_fields(f)
    assert abs(s.diagnostics()["a1"] - a) <= 1e-14


def test_capillary_mode_amplitude_of_the_initial_wave():
    """The tanh profile of the capillary workload (interface y0 + H0 cos 2 pi x,
    c = 1 below) at 128^2: the midpoint sums of the profile reproduce H0."""
    P = W.capillary_64()
    P.m1 = P.m2 = 128
    s = RefSolver(**P.create_kwargs())
    s.set_fields(P.fields())
    assert abs(s.diagnostics()["a1"] - 0.01) <= 1e-12


def test_interface_tips_of_a_piecewise_linear_profile():
    """RT-shaped interface 2 + 0.1 cos(2 pi x) on a periodic 32 x 128 box: the
    highest and lowest c = 1/2 crossings are max and min of the interface
    heights at the cell centres, exactly."""
    m1, m2 = 32, 128
    s = RefSolver(m1, m2, periodic_x=True)
    x = (np.arange(1, m1 + 1) - 0.5) / m1
    yt = 2.0 + 0.1 * np.cos(2 * math.pi * x)
    f = s.zeros()
    f["c"][:] = _linear_interface(s, yt)
    s.set_fields(f)
    d = s.diagnostics()
    assert abs(d["y_top"] - yt.max()) <= 1e-12
    assert abs(d["y_bottom"] - yt.min()) <= 1e-12


def test_interface_tips_count_only_upward_crossings():
    """Light fluid below y = 1, heavy on [1, 2.5], light on [2.5, 3], heavy
    above: upward crossings (light below, heavy above) at 1 and 3; the
    downward one at 2.5 is not a tip."""
    m1, m2 = 8, 128
    h = 1.0 / m1
    s = RefSolver(m1, m2, periodic_x=True)
    y = (np.arange(1, m2 + 1) - 0.5) * h
    w = 4 * h

    def ramp(y0):  # 1 below y0, 0 above, linear over 4 cells
        return np.clip(0.5 - (y - y0) / w, 0.0, 1.0)

    c = ramp(1.0) + (1.0 - ramp(2.5)) * ramp(3.0)
    f = s.zeros()
    f["c"][:] = c[:, None]
    s.set_fields(f)
    d = s.diagnostics()
    assert abs(d["y_top"] - 3.0) <= 1e-12 and abs(d["y_bottom"] - 1.0) <= 1e-12
    f["c"][:] = 0.25
    s.set_fields(f)
    d = s.diagnostics()
    assert d["y_top"] == 0.0 and d["y_bottom"] == m2 * h
