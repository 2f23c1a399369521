"""The single-grid solver's alpha (Sec. 2.1 Step 1: alpha_x = max |u| + c, alpha_y = max |v| + c over the
stage's input state) along a run: against the oracle on the GPU's own states after each stage, bit for bit
the same as a second solver loaded with those states, nodes outside float's range (which the coarse pass
hands to the exact pass) and partial warps at row ends, depth errors in a state set from outside, and a
captured graph that continues from a state set between its launches.
"""
import dataclasses

import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S
from _parity import oracle_grid, oracle_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hw():
    import paper_2208_01260_gb300 as hw
    import torch
    assert torch.cuda.is_available()
    hw.lib()
    return hw


def _oracle_alpha(orc, sc, planes):
    g = oracle_grid(orc, sc)
    p = orc.make_params(eps_w=sc.eps_w)
    _, stat = oracle_state(orc, sc)
    return orc.alpha2d(g, p, [np.ascontiguousarray(a) for a in planes], stat)


@pytest.mark.parametrize("nx,ny,bc", [(203, 37, S.REFLECTIVE), (64, 33, S.PERIODIC), (31, 70, S.OUTFLOW)])
def test_alpha_through_stages(hw, orc, nx, ny, bc):
    """After the initialisation and after each stage: alpha within 1e-14 of the oracle's on the GPU's own
    state, and bit for bit the alpha of a second solver loaded with that state. Row lengths 203 and 31
    leave partial warps."""
    sc = S.hump2d(nx, ny, seed=71, bc=bc)
    s = hw.Solver.from_scenario(sc, hw.make_params())
    t = hw.Solver.from_scenario(sc, hw.make_params())
    dt = s.cfl_dt()
    for k in (0, 1, 2, 3):
        if k:
            s.rk3_stage(k, dt)
        st = s.state()
        a = s.alpha()
        ref = _oracle_alpha(orc, sc, st)
        assert abs(a[0] - ref[0]) <= 1e-14 * ref[0] and abs(a[1] - ref[1]) <= 1e-14 * ref[1], (k, a, ref)
        t.set_state(st)
        assert t.alpha() == a, k
    s.close()
    t.close()


def test_out_of_float_range_nodes_are_evaluated_exactly(hw, orc):
    """A node whose momentum overflows float (alpha_x = |m|/h + c ~ 1e39 decides the maximum) and a node
    whose depth underflows float (on a dry bottom b = 0 there; evaluated, not the maximum): alpha equals
    the oracle's, before and after a stage with dt = 0 (which leaves the state unchanged)."""
    sc = S.hump2d(100, 40, seed=72)
    h, hu, hv, b = sc.h.copy(), sc.hu.copy(), sc.hv.copy(), sc.b.copy()
    hu[17, 45] = 3.0e39  # beyond float's range
    b[30, 90] = 0.0
    h[30, 90] = 1e-40    # below float's normal range, at rest
    hu[30, 90] = hv[30, 90] = 0.0
    sc = dataclasses.replace(sc, h=h, hu=hu, hv=hv, b=b)
    s = hw.Solver.from_scenario(sc, hw.make_params())
    a = s.alpha()
    ref = _oracle_alpha(orc, sc, s.state())
    assert abs(a[0] - ref[0]) <= 1e-14 * ref[0] and abs(a[1] - ref[1]) <= 1e-14 * ref[1], (a, ref)
    assert a[0] > 1e39
    s.rk3_stage(1, 0.0)
    assert s.alpha() == a
    s.close()


def test_depth_errors_of_a_set_state(hw):
    """A negative depth in a state set from outside is reported by the next reduction (hw_alpha, and
    hw_advance before its first stage)."""
    sc = S.hump2d(70, 50, seed=73)
    s = hw.Solver.from_scenario(sc, hw.make_params())
    st = s.state(hw.HW_LAYOUT_PHYSICAL)
    st[0] = st[0].copy()
    st[0][12, 66] = -0.01
    hw.hw_set_state(s.h, st, hw.HW_LAYOUT_PHYSICAL)
    with pytest.raises(hw.HwError) as e:
        s.alpha()
    assert e.value.code == -2
    hw.hw_set_state(s.h, st, hw.HW_LAYOUT_PHYSICAL)
    with pytest.raises(hw.HwError) as e:
        s.advance(2, use_graph=True)
    assert e.value.code == -2
    s.close()


def test_graph_after_set_state(hw):
    """hw_set_state between launches of a captured graph: the run equals the uninterrupted one (spacings
    2^-7 and 2^-6: the state's derivative scalings are exact both ways)."""
    sc = S.hump2d(128, 64, seed=74)
    a = hw.Solver.from_scenario(sc, hw.make_params())
    a.advance(4, use_graph=True)
    st = a.state()
    b = hw.Solver.from_scenario(sc, hw.make_params())
    b.advance(2, use_graph=True)  # b's graph exists; its state is then replaced
    b.set_state(st)
    hw.hw_set_time(b.h, *hw.hw_get_time(a.h))
    a.advance(4, use_graph=True)
    b.advance(4, use_graph=True)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)
    a.close()
    b.close()
