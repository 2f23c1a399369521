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
