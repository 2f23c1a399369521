"""The batched form against the CPU oracle (every instance of a mixed batch, one step at the per-stage
tolerance and several steps at the many-step tolerance, times against the oracle's CFL steps), against
single-grid solvers (same formulas, only the launch organisation differs; the two kernels may contract
multiply-adds differently, so agreement is to rounding), and the autotuner (tile shapes never change
the numbers: bitwise)."""
import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S
from _parity import normwise, oracle_grid, oracle_state, rel_l1, stage_scales, tiny_derivatives

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hw():
    import paper_2208_01260_gb300 as hw
    import torch
    assert torch.cuda.is_available()
    hw.lib()
    return hw


def _mixed_batch():
    sizes = [(64, 64), (100, 37), (257, 130), (33, 301), (150, 150), (2, 5), (513, 70)]
    out = []
    for k, (nx, ny) in enumerate(sizes):
        bc = (S.REFLECTIVE, S.OUTFLOW, S.PERIODIC)[k % 3]
        sc = S.hump2d(nx, ny, seed=100 + k, bc=bc)
        out.append(sc)
    return out


def _oracle_run(orc, sc, nsteps):
    g = oracle_grid(orc, sc)
    p = orc.make_params(eps_w=sc.eps_w)
    cur, stat = oracle_state(orc, sc)
    t = 0.0
    for _ in range(nsteps):
        dt = orc.cfl_dt2d(g, p, cur, stat)
        cur = orc.rk3_step2d(g, p, dt, cur, stat)
        t += dt
    return cur, stat, t


@pytest.mark.parametrize("nsteps,use_graph", [(1, False), (4, True)])
def test_batched_matches_oracle(hw, orc, nsteps, use_graph):
    """Every instance of the mixed batch (all three boundary conditions, a 2x5 grid, ragged x-tiles and
    y-segments) against the oracle's SSP-RK3 steps (Sec. 2.2 eq. RK on the 2D scheme of Sec. 3) at the
    oracle's own CFL time steps (Sec. 4): one step at the per-stage tolerance (normwise 1e-12), four
    steps (two captured graphs) at relative L1 1e-9; the simulated time against the sum of the
    oracle's steps."""
    scs = _mixed_batch()
    b = hw.BatchedSolver(scs)
    b.run(nsteps, use_graph=use_graph)
    t, steps = b.times()
    assert list(steps) == [nsteps] * len(scs)
    for i, sc in enumerate(scs):
        ref, stat, tref = _oracle_run(orc, sc, nsteps)
        got = b.state(i)
        assert abs(t[i] - tref) <= 1e-13 * tref, (i, t[i], tref)
        err = normwise(got, ref, stage_scales(ref, stat))
        if nsteps == 1:
            assert max(err) <= 1e-12, (i, err)
        else:
            assert max(rel_l1(got, ref)) <= 1e-9, (i, rel_l1(got, ref))
            assert max(err) <= 1e-11, (i, err)
    b.close()


@pytest.mark.parametrize("pk", [{"char_decomp": 0}, {"limiter": 0}, {"linear_weights": 1}],
                         ids=["no_char", "no_limiter", "linear_weights"])
def test_batched_matches_oracle_other_parameters(hw, orc, pk):
    """The batched kernels' other instantiations (no characteristic projection, no limiter, linear
    weights) against the oracle with the same parameters, one step at the per-stage tolerance."""
    scs = _mixed_batch()[:5]
    b = hw.BatchedSolver(scs, hw.make_params(**pk))
    b.run(1, use_graph=False)
    for i, sc in enumerate(scs):
        g = oracle_grid(orc, sc)
        p = orc.make_params(eps_w=sc.eps_w, **pk)
        cur, stat = oracle_state(orc, sc)
        dt = orc.cfl_dt2d(g, p, cur, stat)
        ref = orc.rk3_step2d(g, p, dt, cur, stat)
        assert max(normwise(b.state(i), ref, stage_scales(ref, stat))) <= 1e-12, (i, pk)
    b.close()


def test_batched_equals_single_grid_solvers(hw):
    scs = _mixed_batch()
    b = hw.BatchedSolver(scs)
    b.run(5, use_graph=True)
    t, steps = b.times()
    assert list(steps) == [5] * len(scs)
    for i, sc in enumerate(scs):
        s = hw.Solver.from_scenario(sc, hw.make_params())
        ts, n = s.advance(5, use_graph=False)
        assert n == 5 and abs(ts - t[i]) <= 1e-14 * t[i]
        ref = s.state()
        stat = [sc.b, sc.deriv[6], sc.deriv[7]]
        assert max(normwise(b.state(i), ref, stage_scales(ref, stat))) <= 1e-12


def test_batched_fallback_instances_equal_single_grid_solvers(hw):
    """Instances whose derivative data underflow in products (the batched kernels' FP64-pipe
    recomputation of the affected interfaces and nodes) beside ordinary ones."""
    scs = [tiny_derivatives(S.hump2d(70, 45, seed=27)), S.hump2d(64, 64, seed=5),
           tiny_derivatives(S.hump2d(33, 40, seed=28, bc=S.PERIODIC))]
    b = hw.BatchedSolver(scs)
    b.run(3, use_graph=False)
    for i, sc in enumerate(scs):
        s = hw.Solver.from_scenario(sc, hw.make_params())
        s.advance(3, use_graph=False)
        ref = s.state()
        stat = [sc.b, sc.deriv[6], sc.deriv[7]]
        assert max(normwise(b.state(i), ref, stage_scales(ref, stat))) <= 1e-12


def test_tile_shapes_do_not_change_results(hw):
    scs = _mixed_batch()
    a = hw.BatchedSolver(scs)
    c = hw.BatchedSolver(scs)
    for i, sc in enumerate(scs):
        hw.hw_batch_set_tiles(c.h, i, [1, 4, 2][i % 3])
    a.run(3, use_graph=False)
    c.run(3, use_graph=True)
    for i in range(len(scs)):
        for x, y in zip(a.state(i), c.state(i)):
            assert np.array_equal(x, y)


def test_autotuner_picks_valid_tiles(hw, tmp_path):
    from paper_2208_01260_gb300 import autotune
    scs = [S.hump2d(nx, ny, seed=200 + k) for k, (nx, ny) in enumerate([(64, 300), (300, 64), (130, 130)])]
    b = hw.BatchedSolver(scs)
    ref = hw.BatchedSolver(scs)
    res = b.autotune(cache_path=str(tmp_path / "tune.json"))
    assert (tmp_path / "tune.json").exists()
    for i, sc in enumerate(scs):
        assert hw.hw_batch_get_tiles(b.h, i) in autotune.YC_CANDIDATES
    b.run(2)
    ref.run(2)
    for i in range(len(scs)):
        for x, y in zip(b.state(i), ref.state(i)):
            assert np.array_equal(x, y)


def test_config4_full_batch_against_oracle(hw, orc, tmp_path):
    """The benchmark's batched workload at its full size (512 instances, nx and ny log-uniform in [64, 1024],
    58 M points) in the configuration bench.py times (autotuned tiles, two steps from a captured graph): the
    three smallest instances and the largest against the oracle's two SSP-RK3 steps at their own CFL steps,
    every node (relative L1 1e-9, normwise 1e-11), and the times against the oracle's; every instance has
    taken two steps."""
    nxs, nys = S.batch_sizes(512)
    scs = [S.batch_scenario(i, int(nxs[i]), int(nys[i])) for i in range(512)]
    pts = nxs.astype(np.int64) * nys
    b = hw.BatchedSolver(scs)
    b.autotune(cache_path=str(tmp_path / "tune.json"))
    b.run(2, use_graph=True)
    t, steps = b.times()
    assert list(steps) == [2] * 512
    order = np.argsort(pts, kind="stable")
    for i in list(order[:3]) + [int(order[-1])]:
        sc = scs[i]
        ref, stat, tref = _oracle_run(orc, sc, 2)
        got = b.state(int(i))
        assert abs(t[i] - tref) <= 1e-13 * tref, (i, t[i], tref)
        assert max(rel_l1(got, ref)) <= 1e-9, (i, rel_l1(got, ref))
        assert max(normwise(got, ref, stage_scales(ref, stat))) <= 1e-11, i
    b.close()


def test_batch_rejects_bad_grids_and_depth(hw):
    with pytest.raises(hw.HwError):
        hw.hw_batch_create([hw.make_grid(64, 1, dim=1)], hw.make_params())
    sc = S.hump2d(16, 16, seed=3)
    b = hw.hw_batch_create([hw.make_grid(16, 16, 0, 1, 0, 1, 1, 1)], hw.make_params())
    bad = sc.h.copy()
    bad[2, 2] = 0.0
    with pytest.raises(hw.HwError) as e:
        hw.hw_batch_init(b, 0, bad, sc.hu, sc.hv, sc.b, sc.deriv)
    assert e.value.code == -2
    hw.hw_batch_destroy(b)
