"""The paper's examples 4.3, 4.4, 4.5 and 4.9 and the transmissive boundary on the CUDA path, against
the oracle: per stage (1e-12 normwise) on smooth data, at the final time (relative L1 1e-8, the
discontinuous-data bound)."""
import pytest

from paper_2208_01260_gb300 import scenarios as S
from _parity import normwise, oracle_grid, oracle_state, rel_l1, stage_scales

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hw():
    import paper_2208_01260_gb300 as hw
    import torch
    assert torch.cuda.is_available()
    hw.lib()
    return hw


def _pair(hw, orc, sc):
    s = hw.Solver.from_scenario(sc, hw.make_params(eps_w=sc.eps_w))
    g, p = oracle_grid(orc, sc), orc.make_params(eps_w=sc.eps_w)
    st, stat = oracle_state(orc, sc)
    return s, g, p, st, stat


@pytest.mark.parametrize("make", [lambda: S.hump2d(70, 45, seed=27, bc=S.OUTFLOW),
                                  lambda: S.ex44(133)], ids=["hump2d_outflow", "ex44_1d"])
def test_stage_parity_transmissive(hw, orc, make):
    sc = make()
    s, g, p, st, stat = _pair(hw, orc, sc)
    stage = orc.stage2d if sc.dim == 2 else orc.stage1d
    dt = (orc.cfl_dt2d if sc.dim == 2 else orc.cfl_dt1d)(g, p, st, stat)
    cur, base = s.state(), None
    for k in (1, 2, 3):
        s.rk3_stage(k, dt)
        out = s.state()
        oo, bo, _ = stage(g, p, k, dt, cur, stat, base)
        assert max(normwise(out, oo, stage_scales(cur, stat))) <= 1e-12, k
        if k == 1:
            base = s.base()
        cur = out


CASES = [
    ("ex43_large_pulse", lambda: S.ex43(200, 0.2), 0.2),
    ("ex43_small_pulse", lambda: S.ex43(200, 1e-3), 0.2),
    ("ex44", lambda: S.ex44(200), 1.0),
    ("ex45_t15", lambda: S.ex45(200), 15.0),
    ("ex45_t60", lambda: S.ex45(200), 60.0),
    ("ex49", lambda: S.ex49(200), 0.15),
]


@pytest.mark.parametrize("name,make,t_end", CASES, ids=[c[0] for c in CASES])
def test_paper_example_final_time(hw, orc, name, make, t_end):
    sc = make()
    s, g, p, st, stat = _pair(hw, orc, sc)
    run = orc.run1d if sc.dim == 1 else orc.run2d
    out_o, t_o, n_o = run(g, p, st, stat, t_end)
    t, n = s.advance(10 ** 6, t_end=t_end)
    assert n == n_o and abs(t - t_end) <= 1e-14 * t_end
    err = rel_l1(s.state(), out_o)
    assert max(err) <= 1e-8, err


# ------------------------------------------------------------------------------------------------
# Tables 1-3, double rows, through the CUDA path
# ------------------------------------------------------------------------------------------------
import json
import os

import numpy as np

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("step,key", [(False, "table1_ex42_smooth_double"), (True, "table2_ex42_step_double")])
def test_tables_1_2_lake_at_rest_gpu(hw, orc, step, key):
    """Ex. 4.2 (Sec. 4, Tables 1-2): lake at rest over the smooth and the step bottom, N=200, to t=0.5 at
    the CFL step on the device. The residual of h and hu is at the round-off level of the paper's
    double-precision rows, and the final state equals the oracle's run to relative L1 1e-9."""
    sc = S.ex42(200, step=step)
    s, g, p, st, stat = _pair(hw, orc, sc)
    t, n = s.advance(10 ** 6, t_end=0.5)
    assert abs(t - 0.5) <= 1e-14 and n == 166, (t, n)
    out = s.state()
    ref, tref, nref = orc.run1d(g, p, st, stat, 0.5)
    assert nref == n
    gold = GOLD[key]
    e_h, e_m = np.abs(out[0] - 10.0), np.abs(out[1])
    assert e_h.max() < max(100 * gold["h_Linf"], 1e-12) and e_m.max() < max(100 * gold["hu_Linf"], 1e-12)
    assert e_h.mean() < 100 * gold["h_L1"] + 1e-13
    # at rest the oracle's deviation is pure round-off; compare the deviations' sizes, and the states
    assert max(rel_l1(out, ref)[:1]) <= 1e-9
    assert np.abs(out[1] - ref[1]).max() <= max(100 * gold["hu_Linf"], 1e-12)


def test_table_3_lake_at_rest_gpu(hw, orc):
    """Ex. 4.7 (Sec. 4, Table 3): 2D lake at rest, b = 0.8 exp(-50 r^2), periodic, 200x200, t = 0.1. The
    residual of h, hu, hv is at the round-off level of the double row; the state equals the oracle's."""
    sc = S.ex47(200)
    s, g, p, st, stat = _pair(hw, orc, sc)
    t, n = s.advance(10 ** 6, t_end=0.1)
    assert abs(t - 0.1) <= 1e-14
    out = s.state()
    gold = GOLD["table3_ex47_double"]
    eh, em, ew = np.abs(out[0] - 1.0), np.abs(out[1]), np.abs(out[2])
    assert eh.max() < max(100 * gold["h_Linf"], 1e-13)
    assert em.max() < max(100 * gold["hu_Linf"], 1e-13) and ew.max() < max(100 * gold["hv_Linf"], 1e-13)
    assert eh.mean() < 100 * gold["h_L1"] + 1e-15
    ref, tref, nref = orc.run2d(g, p, st, stat, 0.1)
    assert nref == n
    assert rel_l1(out, ref)[0] <= 1e-9
