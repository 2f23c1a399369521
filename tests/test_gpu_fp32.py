"""The single-precision variant (params.precision = HW_FP32; the paper's single-precision runs of
Sec. 4, Tables 1-3) against the oracle computing every operation in float, and against the double
oracle. Tolerance: per stage and for the RHS, 2e-5 normwise (about 330 float unit round-offs; the
float oracle itself differs from the double one by at most 35 of them on these cases, and the GPU
rearranges the same formulas as in double, where 1e-12 is about 9000 double round-offs)."""
import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S
from _parity import normwise, oracle_grid, oracle_state, rel_l1, rhs_scales, stage_scales

pytestmark = pytest.mark.gpu
TOL32 = 2e-5


@pytest.fixture(scope="module")
def hw():
    import paper_2208_01260_gb300 as hw
    import torch
    assert torch.cuda.is_available()
    hw.lib()
    return hw


def _solver32(hw, sc, **pk):
    return hw.Solver.from_scenario(sc, hw.make_params(eps_w=sc.eps_w, precision=hw.HW_FP32, **pk))


CASES = [
    ("hump_reflective", lambda: S.hump2d(70, 45, seed=21)),
    ("strip_reflective", lambda: S.bumps2d(150, 80, strip=0.01)),
    ("hump_periodic", lambda: S.hump2d(131, 67, seed=22, bc=S.PERIODIC)),
    ("ex49_outflow", lambda: S.ex49(64)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp32_rhs_and_stages(hw, orc, name, make):
    sc = make()
    s = _solver32(hw, sc)
    g, p = oracle_grid(orc, sc), orc.make_params(eps_w=sc.eps_w)
    st, stat = oracle_state(orc, sc)
    st32 = [np.asarray(a, dtype=np.float32).astype(np.float64) for a in st]
    R = s.rhs()
    R32, _ = orc.rhs2d(g, p, st32, stat, single=True)
    R64, _ = orc.rhs2d(g, p, st, stat)
    sc_r = rhs_scales(st, stat, min(sc.dx, sc.dy))
    assert max(normwise(R, R32, sc_r)) <= TOL32
    assert max(normwise(R, R64, sc_r)) <= TOL32
    dt = orc.cfl_dt2d(g, p, st, stat)
    cur, base = s.state(), None
    for k in (1, 2, 3):
        s.rk3_stage(k, dt)
        out = s.state()
        oo, _, _ = orc.stage2d(g, p, k, dt, cur, stat, base, single=True)
        assert max(normwise(out, oo, stage_scales(cur, stat))) <= TOL32, k
        if k == 1:
            base = s.base()
        cur = out
    # the state really is float: eta, m, w come back unconverted and are exact single-precision values
    for a in s.state()[:3]:
        assert np.array_equal(a, a.astype(np.float32).astype(np.float64))


def test_fp32_lake_at_rest_ex47(hw, orc):
    """Ex. 4.7 (200x200, t = 0.1) in single precision: the residual of h is at the level of Table 3's
    single row and of the float oracle's run (round-off, not truncation)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    sgl = gold["table3_ex47_single"]
    sc = S.ex47(200)
    s = _solver32(hw, sc)
    t, n = s.advance(10 ** 6, t_end=0.1)
    out = s.state()
    h_l1 = np.abs(out[0] - 1.0).mean()
    m_li = max(np.abs(out[1]).max(), np.abs(out[2]).max())
    assert 0.0 < h_l1 < 100 * sgl["h_L1"] and m_li < 100 * sgl["hu_Linf"]
    g, p = oracle_grid(orc, sc), orc.make_params()
    st, stat = oracle_state(orc, sc)
    res, steps = orc.lake_run(g, p, st, stat, 0.1, "single")
    assert steps == n
    assert res[0] / 30 < h_l1 < 30 * res[0]


def test_fp32_final_time_against_double(hw, orc):
    """The benchmark's strip over bumps (150x80, reflective) to t = 0.05: the float run stays within the
    float round-off budget of the double oracle's: relative L1 of (eta, m, w) <= 2e-6, and normwise on
    the stage scales <= 1e-4 for every group (the derivative groups are nearly zero over much of the
    domain, so their relative L1 says little)."""
    sc = S.bumps2d(150, 80, strip=0.01)
    s = _solver32(hw, sc)
    g, p = oracle_grid(orc, sc), orc.make_params()
    st, stat = oracle_state(orc, sc)
    out_o, t_o, n_o = orc.run2d(g, p, st, stat, 0.05)
    t, n = s.advance(10 ** 6, t_end=0.05)
    assert n == n_o
    out = s.state()
    err = rel_l1(out, out_o)
    nw = normwise(out, out_o, stage_scales(st, stat))
    assert err[0] <= 2e-6 and max(nw) <= 1e-4, (err, nw)


def test_fp32_graph_matches_eager(hw):
    sc = S.hump2d(100, 77, seed=41)
    a, b = _solver32(hw, sc), _solver32(hw, sc)
    a.advance(6, use_graph=True)
    b.advance(6, use_graph=False)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)


def test_fp32_restrictions(hw):
    """Single precision is for 2D single-grid solvers: 1D, the batched form and the adjoint refuse it."""
    from paper_2208_01260_gb300 import adjoint as A
    p32 = hw.make_params(precision=hw.HW_FP32)
    with pytest.raises(hw.HwError):
        hw.Solver(hw.make_grid(64), p32)
    with pytest.raises(hw.HwError):
        hw.BatchedSolver([S.hump2d(40, 40, seed=3)], params=p32)
    sc = S.hump2d(40, 33, seed=5)
    s = _solver32(hw, sc)
    import torch
    lam = [torch.zeros(sc.ny, sc.nx, dtype=torch.float64, device="cuda") for _ in range(12)]
    with pytest.raises(hw.HwError):
        A.hw_adjoint_step(s.h, 1e-4, lam[:9], lam[9:])
