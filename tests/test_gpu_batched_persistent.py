"""The batched form's persistent step (one cooperative launch per SSP-RK3 step, phases separated by bounded
grid barriers) against the CPU oracle and against the per-phase form, mode switches in the middle of a
run, the other kernel instantiations, and the bounded barrier wait itself (a block that never arrives:
the others' waits run out, every block leaves, the host reads HW_ERR_TIMEOUT and the batch stays
usable)."""
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
    return [S.hump2d(nx, ny, seed=100 + k, bc=(S.REFLECTIVE, S.OUTFLOW, S.PERIODIC)[k % 3])
            for k, (nx, ny) in enumerate(sizes)]


def _oracle_run(orc, sc, nsteps, **pk):
    g = oracle_grid(orc, sc)
    p = orc.make_params(eps_w=sc.eps_w, **pk)
    cur, stat = oracle_state(orc, sc)
    t = 0.0
    for _ in range(nsteps):
        dt = orc.cfl_dt2d(g, p, cur, stat)
        cur = orc.rk3_step2d(g, p, dt, cur, stat)
        t += dt
    return cur, stat, t


def test_persistent_launch_shape(hw):
    import torch
    b = hw.BatchedSolver(_mixed_batch()[:2], persistent=True)
    on, blocks = hw.hw_batch_get_persistent(b.h)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert on and blocks >= sms and blocks % sms == 0, (blocks, sms)
    b.set_persistent(False)
    assert not b.persistent
    b.close()


@pytest.mark.parametrize("nsteps,use_graph", [(1, False), (4, True)])
def test_persistent_matches_oracle(hw, orc, nsteps, use_graph):
    """Every instance of the mixed batch against the oracle's SSP-RK3 steps (Sec. 2.2 eq. RK, 2D scheme of
    Sec. 3) at the oracle's CFL steps (Sec. 4): one step at the per-stage tolerance (normwise 1e-12), four
    steps (two graphs of two launches) at relative L1 1e-9; times against the sum of the oracle's steps."""
    scs = _mixed_batch()
    b = hw.BatchedSolver(scs, persistent=True)
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


def test_persistent_equals_per_phase_form(hw):
    """Same source for every phase, so the same numbers: the states and times of the two forms are equal
    bit for bit, over eager steps, graph steps and a switch of form in the middle of the run (which must
    hand over the current plane set and time)."""
    scs = _mixed_batch()
    a = hw.BatchedSolver(scs)
    c = hw.BatchedSolver(scs, persistent=True)
    a.run(7, use_graph=True)
    c.run(1, use_graph=False)
    c.run(2, use_graph=True)
    c.set_persistent(False)
    c.run(1, use_graph=False)  # odd step count: the per-phase form continues from the other plane set
    c.set_persistent(True)
    c.run(3, use_graph=True)  # a graph of two steps plus one eager step
    ta, na = a.times()
    tc, nc = c.times()
    assert list(na) == list(nc) == [7] * len(scs)
    assert np.array_equal(ta, tc)
    for i in range(len(scs)):
        for q, (x, y) in enumerate(zip(a.state(i), c.state(i))):
            assert np.array_equal(x, y), (i, q, float(np.abs(x - y).max()))
    a.close()
    c.close()


@pytest.mark.parametrize("pk", [{"char_decomp": 0}, {"limiter": 0}, {"linear_weights": 1}],
                         ids=["no_char", "no_limiter", "linear_weights"])
def test_persistent_other_parameters(hw, orc, pk):
    """The step kernel's other instantiations against the oracle with the same parameters (one step at the
    per-stage tolerance) and against the per-phase form (bitwise, two steps)."""
    scs = _mixed_batch()[:5]
    params = hw.make_params(**pk)
    b = hw.BatchedSolver(scs, params, persistent=True)
    b.run(1, use_graph=False)
    for i, sc in enumerate(scs):
        ref, stat, _ = _oracle_run(orc, sc, 1, **pk)
        assert max(normwise(b.state(i), ref, stage_scales(ref, stat))) <= 1e-12, (i, pk)
    b.run(1, use_graph=False)
    a = hw.BatchedSolver(scs, params)
    a.run(2, use_graph=False)
    for i in range(len(scs)):
        for x, y in zip(a.state(i), b.state(i)):
            assert np.array_equal(x, y), (i, pk)
    a.close()
    b.close()


def test_persistent_fallback_instances(hw):
    """Instances whose products leave the integer fast path (FP64-pipe recomputation of the affected
    interfaces and nodes) beside ordinary ones: as the per-phase form, bit for bit."""
    scs = [tiny_derivatives(S.hump2d(70, 45, seed=27)), S.hump2d(64, 64, seed=5),
           tiny_derivatives(S.hump2d(33, 40, seed=28, bc=S.PERIODIC))]
    a = hw.BatchedSolver(scs)
    b = hw.BatchedSolver(scs, persistent=True)
    a.run(3, use_graph=False)
    b.run(3, use_graph=False)
    for i in range(len(scs)):
        for x, y in zip(a.state(i), b.state(i)):
            assert np.array_equal(x, y)
    a.close()
    b.close()


def test_bounded_barrier_wait(hw):
    """Block 0 of one step launch leaves before the first grid barrier: the other blocks' waits run out
    (2 ms bound), every block leaves, the call returns HW_ERR_TIMEOUT, and the batch then steps normally
    from its unchanged state (equal to a batch that never saw the failed launch)."""
    scs = _mixed_batch()[:3]
    b = hw.BatchedSolver(scs, persistent=True)
    ref = hw.BatchedSolver(scs, persistent=True)
    b.run(1, use_graph=False)
    ref.run(1, use_graph=False)
    assert hw.hw_batch_test_barrier_timeout(b.h) == -5
    t0, n0 = b.times()
    assert list(n0) == [1] * len(scs)
    b.run(2, use_graph=True)
    ref.run(2, use_graph=True)
    assert np.array_equal(b.times()[0], ref.times()[0])
    for i in range(len(scs)):
        for x, y in zip(b.state(i), ref.state(i)):
            assert np.array_equal(x, y)
    b.set_persistent(False)
    assert hw.hw_batch_test_barrier_timeout(b.h) == -5  # the hook runs the step kernel regardless of the form
    b.close()
    ref.close()
