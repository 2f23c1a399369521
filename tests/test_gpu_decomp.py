"""Block decomposition of one grid on the GPU against the undecomposed solver, bit for bit.

Every block computes its interfaces and nodes from the same values in the same arithmetic as the
undecomposed grid once its 2-node ring is refreshed (hwswe.h, block decomposition), and alpha is the
maximum over the blocks (Sec. 2.1 Step 1), so the states must be equal in every bit, at every step,
for every split and boundary condition: any ring node taken from the wrong place, a corner missed, a
parity sign wrong or an alpha taken from one block only shows up as a difference.
"""
import dataclasses

import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hw():
    import paper_2208_01260_gb300 as hw
    import torch
    assert torch.cuda.is_available()
    hw.lib()
    return hw


def _scenario(nx, ny, bcx, bcy, seed):
    sc = S.hump2d(nx, ny, seed=seed, bc=bcx, hump_max=0.05)
    return dataclasses.replace(sc, bc_y=bcy)


CASES = [
    ("reflective_2x2", 203, 121, S.REFLECTIVE, S.REFLECTIVE, 2, 2),
    ("periodic_4x2", 203, 121, S.PERIODIC, S.PERIODIC, 4, 2),
    ("outflow_4x2", 150, 97, S.OUTFLOW, S.OUTFLOW, 4, 2),
    ("mixed_2x2", 130, 70, S.PERIODIC, S.REFLECTIVE, 2, 2),
    ("mixed_4x2", 130, 70, S.REFLECTIVE, S.OUTFLOW, 4, 2),
    ("periodic_1x3", 66, 90, S.PERIODIC, S.PERIODIC, 1, 3),
]


@pytest.mark.parametrize("name,nx,ny,bcx,bcy,px,py", CASES, ids=[c[0] for c in CASES])
def test_decomposed_equals_undecomposed(hw, name, nx, ny, bcx, bcy, px, py):
    sc = _scenario(nx, ny, bcx, bcy, seed=61)
    ref = hw.Solver.from_scenario(sc, hw.make_params())
    dd = hw.DecomposedSolver(sc, px, py)
    for chunk, graph in ((1, False), (1, False), (6, True), (12, False)):  # 20 steps; graph and eager paths
        t1, n1 = ref.advance(chunk, use_graph=graph)
        t2, n2 = dd.advance(chunk, use_graph=graph)
        assert n1 == n2 == chunk and t1 == t2
        for q, (a, b) in enumerate(zip(ref.state(), dd.state())):
            assert np.array_equal(a, b), (name, q, float(np.abs(a - b).max()))
    dd.close()
    ref.close()


def test_decomposed_end_time_and_depth_error(hw):
    sc = _scenario(96, 64, S.REFLECTIVE, S.PERIODIC, seed=62)
    ref = hw.Solver.from_scenario(sc, hw.make_params())
    dd = hw.DecomposedSolver(sc, 2, 2)
    t1, n1 = ref.advance(10 ** 6, t_end=0.01)
    t2, n2 = dd.advance(10 ** 6, t_end=0.01)
    assert (t1, n1) == (t2, n2) and abs(t1 - 0.01) < 1e-15
    for a, b in zip(ref.state(), dd.state()):
        assert np.array_equal(a, b)
    bad = dataclasses.replace(sc, h=sc.h.copy())
    bad.h[40, 70] = -0.1
    g = hw.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y, dim=2)
    d = hw.hw_dd_create(g, hw.make_params(), 2, 2)
    arrs = [np.ascontiguousarray(a) for a in [bad.h, bad.hu, bad.hv, bad.b] + list(bad.deriv)]
    with pytest.raises(hw.HwError) as e:
        hw.hw_dd_init(d, arrs[0], arrs[1], arrs[2], arrs[3], arrs[4:])
    assert e.value.code == -2
    hw.hw_dd_destroy(d)


def test_decomposed_full_size(hw):
    """The benchmark workload (2048^2, reflective, 8 bumps + strip) in 2 x 2 blocks, 6 steps from graphs."""
    sc = S.bumps2d(2048, 2048, strip=0.01)
    ref = hw.Solver.from_scenario(sc, hw.make_params())
    ref.advance(6)
    a = ref.state()
    ref.close()
    dd = hw.DecomposedSolver(sc, 2, 2)
    dd.advance(6)
    b = dd.state()
    dd.close()
    for q in range(9):
        assert np.array_equal(a[q], b[q]), q


def test_protocol_in_one_process_with_cuda_blocks(hw):
    """The multi-process protocol (paper_2208_01260_gb300.decomp) with the library's CUDA block solvers,
    all 2 x 3 blocks in this process (world size 1: every strip stays on the GPU), against the
    undecomposed solver."""
    from paper_2208_01260_gb300 import decomp
    sc = _scenario(101, 77, S.REFLECTIVE, S.PERIODIC, seed=63)
    g = hw.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y, dim=2)
    params = hw.make_params()
    plan = decomp.Plan(g, 2, 3, 1)
    comm = decomp.Comm(0, 1)
    blocks = {p: decomp.CudaBlock(g, params, 2, 3, p) for p in plan.local_parts(0)}
    decomp.initialise(blocks, plan, comm, lambda p: decomp.window12(sc, plan.info[p]))
    ref = hw.Solver.from_scenario(sc, params)
    for _ in range(4):
        decomp.rk3_step(blocks, plan, comm)
        ref.advance(1, use_graph=False)
    got = decomp.gather(plan, {p: b.state() for p, b in blocks.items()})
    for q, (a, b) in enumerate(zip(ref.state(), got)):
        assert np.array_equal(a, b), (q, float(np.abs(a - b).max()))
    for b in blocks.values():
        b.close()
