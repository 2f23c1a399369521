"""The paper's remaining examples through the oracle (Sec. 4: Ex. 4.3, 4.4, 4.5, 4.9) and the
transmissive boundary they use (the paper names none; the reading here copies the boundary node into
the ghosts). Pins: what the mathematics fixes (uniform flow is a steady solution, the lake at rest is
kept, mirror symmetry) and what the paper states about the flows (wave speeds, undisturbed far field)."""
import math

import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S
from test_oracle_scheme import grid_of, state_of


def _uniform(dim, bc, n=24):
    """Flat bottom, h = 1, u = 0.5 (v = -0.3 in 2D): a steady solution of the equations."""
    if dim == 1:
        z = np.zeros(n)
        return S.Scenario(1, n, 1, 0.0, 1.0, 0.0, 1.0, bc, S.PERIODIC, np.ones(n), 0.5 * np.ones(n), z.copy(),
                          [z.copy(), z.copy(), z.copy()])
    z = np.zeros((n, n + 3))
    return S.Scenario(2, n + 3, n, 0.0, 1.0, 0.0, 1.0, bc, bc, np.ones_like(z), 0.5 + z, z.copy(),
                      [z.copy() for _ in range(8)], hv=-0.3 + z)


@pytest.mark.parametrize("dim", [1, 2])
def test_uniform_flow_passes_transmissive_boundaries(orc, dim):
    sc = _uniform(dim, S.OUTFLOW)
    g, p = grid_of(orc, sc), orc.make_params()
    st, stat = state_of(orc, sc)
    run = orc.run1d if dim == 1 else orc.run2d
    out, t, n = run(g, p, st, stat, 0.1)
    assert n > 5
    for a, b in zip(out, st):
        assert np.abs(a - b).max() <= 1e-13
    # walls instead would stop the flow at the boundary: the check above is not vacuous
    sc = _uniform(dim, S.REFLECTIVE)
    g = grid_of(orc, sc)
    st, stat = state_of(orc, sc)
    out, t, n = run(g, p, st, stat, 0.1)
    assert np.abs(out[1] - st[1]).max() > 1e-2


def test_lake_at_rest_with_transmissive_boundaries(orc):
    sc = S.bumps2d(40, 30, strip=0.0, bc=S.OUTFLOW)
    g, p = grid_of(orc, sc), orc.make_params()
    st, stat = state_of(orc, sc)
    cur = st
    for _ in range(10):
        cur = orc.rk3_step2d(g, p, orc.cfl_dt2d(g, p, cur, stat), cur, stat)
    assert max(np.abs(cur[0] - 1).max(), np.abs(cur[1]).max(), np.abs(cur[2]).max()) < 1e-12


@pytest.mark.parametrize("eps", [0.2, 1e-3])
def test_ex43_pulse_splits_at_the_characteristic_speeds(orc, eps):
    """Ex. 4.3: the pulse on [1.1, 1.2] splits into waves moving at -+sqrt(g h); at t = 0.2 the left
    wave's crest sits near 1.15 - 0.2 sqrt(g) (depth 1 there; the large pulse runs ahead of that linear
    speed, as a nonlinear wave on deeper water), carrying half the pulse, and the surface right of the
    bump has risen (the right wave has passed it)."""
    sc = S.ex43(200, eps)
    g, p = grid_of(orc, sc), orc.make_params(eps_w=sc.eps_w)
    st, stat = state_of(orc, sc)
    out, t, n = orc.run1d(g, p, st, stat, 0.2)
    x = S.axis(sc.nx, sc.x0, sc.x1, sc.bc_x)
    left = x < 1.1
    crest = x[left][np.argmax(out[0][left])]
    linear = 1.15 - 0.2 * math.sqrt(9.812)
    if eps < 0.01:
        assert abs(crest - linear) < 0.03
    else:
        assert linear - 0.1 < crest < linear
    assert (out[0][left].max() - 1.0) == pytest.approx(eps / 2, rel=0.25)
    assert (out[0][x > 1.6].max() - 1.0) > 0.2 * eps


def test_ex44_far_field_is_undisturbed(orc):
    """Ex. 4.4 to t = 1: the rarefaction and the shocks stay inside (-10, 10), so the transmissive
    boundaries keep the initial far-field states exactly (walls would reflect the inflow u = 1)."""
    sc = S.ex44(200)
    g, p = grid_of(orc, sc), orc.make_params()
    st, stat = state_of(orc, sc)
    out, t, n = orc.run1d(g, p, st, stat, 1.0)
    assert abs(out[0][0] - 2.0) < 1e-12 and abs(out[1][0] - 2.0) < 1e-12
    assert abs(out[0][-1] - 0.35) < 1e-12 and abs(out[1][-1]) < 1e-12
    assert out[1].max() > 2.5  # the shock over the bump carries more discharge than the inflow


def test_ex45_dam_break_reaches_the_boundaries_only_late(orc):
    """Ex. 4.5: at t = 15 the waves (speed about sqrt(9.812 x 20) = 14) are still inside (0, 1500); by
    t = 60 they have left through both transmissive boundaries, which then carry flow out."""
    sc = S.ex45(200)
    g, p = grid_of(orc, sc), orc.make_params()
    st, stat = state_of(orc, sc)
    out, t, n = orc.run1d(g, p, st, stat, 15.0)
    assert out[0][0] == pytest.approx(20.0, abs=1e-12) and out[0][-1] == pytest.approx(15.0, abs=1e-12)
    assert abs(out[1][0]) < 1e-12 and abs(out[1][-1]) < 1e-12
    out, t, n = orc.run1d(g, p, st, stat, 60.0)
    assert out[0][0] < 20.0 - 0.1 and out[1][0] > 1.0 and out[1][-1] > 1.0


def test_ex49_is_symmetric_about_y_equals_one(orc):
    """Ex. 4.9 (80x80 to t = 0.15): the data are symmetric about y = 1, so eta and hu are even and hv is
    odd under y -> 2 - y, to rounding (the initial data are discontinuous, so not bitwise)."""
    sc = S.ex49(80)
    g, p = grid_of(orc, sc), orc.make_params()
    st, stat = state_of(orc, sc)
    out, t, n = orc.run2d(g, p, st, stat, 0.15)
    assert np.abs(out[0] - out[0][::-1, :]).max() < 1e-13
    assert np.abs(out[1] - out[1][::-1, :]).max() < 1e-13
    assert np.abs(out[2] + out[2][::-1, :]).max() < 1e-13
    assert out[0].max() < 1.1 and out[0].min() > 0.4  # the column has collapsed and spread
