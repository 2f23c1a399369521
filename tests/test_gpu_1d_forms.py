"""The 1D kernels' two forms at the grid sizes where the library switches between them.

Small 1D grids run the sweep with each interface spread over four lanes (while the grid has at most 4864
interfaces) and the node update with each node over two lanes (at most 9728 nodes); larger grids run one
thread per interface and per node. Both sides of each switch are held to the oracle here, the right-hand
side and the three stages of a step, at the per-stage tolerance of the other parity tests, together
with grids of 2, 3 and 33 nodes, whose last warps hold lanes past the grid's end.

The derivative equations' right-hand side is a difference of interface values that are themselves
difference quotients of the fluxes, divided by dx, so its rounding grows like 1/dx^2 and, at thousands of
nodes, exceeds 1e-12 of the groups' scales in the stages too (U stays near 1e-15). A group is therefore
held to 1e-12 or to ten times the oracle's own change when eta moves by one unit in the last place at
every node, whichever is larger (the reading the full-size final-time test takes for its near-zero group).
"""
import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S
from _parity import normwise, oracle_grid, oracle_state, rhs_scales, stage_scales

pytestmark = pytest.mark.gpu

SIZES = [2, 3, 33, 4863, 4864, 9728, 9729]


def _ulp(state):
    """The state with eta moved by one unit in the last place at every node (seeded random signs)."""
    r = np.random.default_rng(3)
    out = [np.array(a, copy=True) for a in state]
    out[0] = out[0] * (1.0 + r.choice([-1.0, 1.0], out[0].shape) * 2.0 ** -52)
    return out


def _within(err, sens, what=None):
    for e, o in zip(err, sens):
        assert e <= max(1e-12, 10.0 * o), (what, err, sens)


@pytest.mark.parametrize("nx", SIZES)
def test_1d_forms_against_oracle(nx, orc):
    import paper_2208_01260_gb300 as hw
    sc = S.perturbed1d(n=nx, perturb=0.05) if nx < 100 else S.accuracy1d(nx)
    s = hw.Solver.from_scenario(sc, hw.make_params(eps_w=sc.eps_w))
    g, p = oracle_grid(orc, sc), orc.make_params(eps_w=sc.eps_w)
    st, stat = oracle_state(orc, sc)
    R = s.rhs()
    Ro, al = orc.rhs1d(g, p, st, stat)
    assert abs(s.alpha()[0] - al) <= 1e-14 * al
    sc_r = rhs_scales(st, stat, sc.dx)
    sens = normwise(orc.rhs1d(g, p, _ulp(st), stat)[0], Ro, sc_r)
    _within(normwise(R, Ro, sc_r), sens)
    dt = orc.cfl_dt1d(g, p, st, stat)
    assert abs(s.cfl_dt() - dt) <= 1e-14 * dt
    cur, base = s.state(), None
    for k in (1, 2, 3):
        s.rk3_stage(k, dt)
        got = s.state()
        ref, base_orc, _ = orc.stage1d(g, p, k, dt, cur, stat, base)
        ref2, base_orc2, _ = orc.stage1d(g, p, k, dt, _ulp(cur), stat, base)
        scl = stage_scales(cur, stat)
        _within(normwise(got, ref, scl), normwise(ref2, ref, scl), k)
        if k == 1:  # the step's base: U^n and the limited derivatives V^{n,mod}
            base = s.base()
            _within(normwise(base, base_orc, scl), normwise(base_orc2, base_orc, scl), "base")
        cur = got
    # a run of the graph to an end time stays finite and moves the clock exactly there
    t, n = s.advance(10 ** 6, t_end=2 * dt + 0.5 * dt)
    assert n >= 1 and abs(t - 2.5 * dt) <= 1e-12 * dt * 10
    assert all(np.all(np.isfinite(x)) for x in s.state())
    s.close()
