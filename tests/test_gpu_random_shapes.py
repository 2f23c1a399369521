"""Every RK stage of the CUDA path against the oracle on seeded random grid shapes.

The sweeps run over flattened extended lines (x: rows of nx + 4 nodes cut into tiles of 189 interfaces;
y: groups of 2 columns, ny + 4 rows each, cut into tiles of 93 interfaces, a single column in the last
group when nx is odd), so where a tile boundary falls inside a row or a column, and which rows a tile
spans, depends on nx and ny. These cases draw nx and ny log-uniformly (seeded) with every boundary
condition, on smooth data (a Gaussian surface hump over Gaussian bumps) and on data with a jump (the
benchmark's perturbation strip, reflective walls), and hold each stage to the per-stage tolerance of
the other parity tests.
"""
import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S
from _parity import normwise, oracle_grid, oracle_state, stage_scales

pytestmark = pytest.mark.gpu

SEED = S.SEED_BASE + 77


def _shapes(count, lo, hi, seed):
    r = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        nx, ny = (int(v) for v in np.exp(r.uniform(np.log(lo), np.log(hi), 2)))
        if nx * ny <= 120_000:
            out.append((nx, ny))
    return out


SMOOTH = [(nx, ny, bc) for (nx, ny), bc in zip(_shapes(12, 2, 700, SEED), [S.PERIODIC, S.REFLECTIVE, S.OUTFLOW] * 4)]
JUMP = _shapes(6, 8, 700, SEED + 1)


def _stages(hw, orc, sc):
    s = hw.Solver.from_scenario(sc, hw.make_params(eps_w=sc.eps_w))
    g, p = oracle_grid(orc, sc), orc.make_params(eps_w=sc.eps_w)
    st, stat = oracle_state(orc, sc)
    dt = orc.cfl_dt2d(g, p, st, stat)
    assert abs(s.cfl_dt() - dt) <= 1e-14 * dt
    cur, base = s.state(), None
    for k in (1, 2, 3):
        s.rk3_stage(k, dt)
        got = s.state()
        ref, base_orc, _ = orc.stage2d(g, p, k, dt, cur, stat, base)
        err = normwise(got, ref, stage_scales(cur, stat))
        assert max(err) <= 1e-12, (sc.nx, sc.ny, k, err)
        if k == 1:
            base = s.base()
            assert max(normwise(base, base_orc, stage_scales(cur, stat))) <= 1e-12
        cur = got
    s.close()


@pytest.mark.parametrize("nx,ny,bc", SMOOTH, ids=["%dx%d_bc%d" % c for c in SMOOTH])
def test_random_shape_smooth(nx, ny, bc, orc):
    import paper_2208_01260_gb300 as hw
    _stages(hw, orc, S.hump2d(nx, ny, seed=SEED + nx * 1000 + ny, bc=bc))


@pytest.mark.parametrize("nx,ny", JUMP, ids=["%dx%d" % c for c in JUMP])
def test_random_shape_strip(nx, ny, orc):
    import paper_2208_01260_gb300 as hw
    _stages(hw, orc, S.bumps2d(nx, ny, strip=0.01))
