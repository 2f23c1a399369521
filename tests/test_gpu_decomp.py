"""Block decomposition of one grid on the GPU against the undecomposed solver, bit for bit.

Every block computes its interfaces and nodes from the same values in the same arithmetic as the
undecomposed grid once its 2-node ring is refreshed (hwswe.h, block decomposition), and alpha is the
maximum over the blocks (Sec. 2.1 Step 1), so the states must be equal in every bit, at every step,
for every split and boundary condition: any ring node taken from the wrong place, a corner missed, a
parity sign wrong or an alpha taken from one block only shows up as a difference.
"""
import dataclasses
import os
import socket
import sys

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


@pytest.mark.parametrize("pk", [{"char_decomp": 0, "limiter": 0}, {"linear_weights": 1}], ids=["no_char_no_limiter", "linear"])
def test_decomposed_equals_undecomposed_other_parameters(hw, pk):
    """The other kernel instantiations through the blocks: still bitwise."""
    sc = _scenario(90, 70, S.REFLECTIVE, S.PERIODIC, seed=65)
    params = hw.make_params(**pk)
    ref = hw.Solver.from_scenario(sc, params)
    dd = hw.DecomposedSolver(sc, 3, 2, params)
    ref.advance(5)
    dd.advance(5)
    for a, b in zip(ref.state(), dd.state()):
        assert np.array_equal(a, b)
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


@pytest.mark.parametrize("bcx,bcy,px,py", [(S.REFLECTIVE, S.REFLECTIVE, 2, 2), (S.PERIODIC, S.PERIODIC, 4, 2),
                                           (S.OUTFLOW, S.REFLECTIVE, 2, 1), (S.PERIODIC, S.REFLECTIVE, 1, 3)],
                         ids=["reflective_2x2", "periodic_4x2", "outflow_reflective_2x1", "periodic_reflective_1x3"])
def test_decomposed_adjoint_equals_undecomposed(hw, orc, bcx, bcy, px, py):
    """The gauge-misfit gradient over the blocks (hw_dd_adjoint_run: each block reverses its own stages, the
    transpose of the halo exchange returns ring adjoints to their owners, the alpha adjoint is applied
    once) against the undecomposed adjoint on its whole-run tape, and against the oracle's forward-mode
    dual numbers along three random directions. The loss is equal bit for bit (the forward runs are
    equal). The gradients differ by the order of the atomic sums, whose rounding scales with the adjoint
    state (the gradient of b is a near-cancelling sum of terms of that size): they are held to 1e-10 of the
    largest state-gradient entry, against differences of 1e-15..1e-14 measured (the undecomposed adjoint
    on its tape and with checkpointing differs by as much), while a lost ring or alpha contribution would
    be of the order of the adjoint itself."""
    import torch
    from paper_2208_01260_gb300 import adjoint as A
    sc = _scenario(96, 66, bcx, bcy, seed=64)
    nsteps, ng = 5, 9
    ref = hw.Solver.from_scenario(sc, hw.make_params())
    dts = [ref.cfl_dt()] * nsteps
    rng = np.random.default_rng(8)
    gidx = rng.choice(sc.nx * sc.ny, ng, replace=False).astype(np.int32)
    obs = 1.0 + 0.002 * rng.normal(size=nsteps * ng)
    gs = torch.empty(9, sc.ny, sc.nx, dtype=torch.float64, device="cuda")
    gb = torch.empty(3, sc.ny, sc.nx, dtype=torch.float64, device="cuda")
    loss, _ = A.hw_adjoint_run(ref.h, dts, gidx, obs, A.HW_ADJ_TAPE, [gs[q] for q in range(9)],
                               [gb[q] for q in range(3)])
    ref.close()
    dd = hw.DecomposedSolver(sc, px, py)
    ds, db = torch.full_like(gs, float("nan")), torch.full_like(gb, float("nan"))
    loss_dd = hw.hw_dd_adjoint_run(dd.h, dts, gidx, obs, [ds[q] for q in range(9)], [db[q] for q in range(3)])
    # a second run from the unchanged block states gives the same
    ds2, db2 = torch.empty_like(gs), torch.empty_like(gb)
    loss_dd2 = hw.hw_dd_adjoint_run(dd.h, dts, gidx, obs, [ds2[q] for q in range(9)], [db2[q] for q in range(3)])
    dd.close()
    assert loss_dd == loss and loss_dd2 == loss
    scale = float(gs.abs().max())
    for got, want in ((ds, gs), (db, gb), (ds2, gs), (db2, gb)):
        assert torch.isfinite(got).all()
        err = float((got - want).abs().max())
        assert err <= 1e-10 * scale, (err, scale)
    g = orc.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y)
    st, stat = orc.to_state2d(sc.h, sc.hu, sc.hv, sc.b, sc.deriv)
    D = np.concatenate([ds.cpu().numpy(), db.cpu().numpy()])
    for seed in (1, 2, 3):
        r = np.random.default_rng(seed)
        dst = [r.normal(size=(sc.ny, sc.nx)) * 1e-3 for _ in range(9)]
        dstat = [r.normal(size=(sc.ny, sc.nx)) * 1e-3 for _ in range(3)]
        L, dL = orc.gauge_loss_dual2d(g, orc.make_params(), st, stat, dst, dstat, dts, gidx, obs)
        assert abs(L - loss) <= 1e-10 * abs(L)
        gv = float((D * np.concatenate([np.stack(dst), np.stack(dstat)])).sum())
        assert abs(gv - dL) <= 1e-8 * abs(dL), (gv, dL)


def _gpu_rank(rank, ws, port, q):
    """One rank of the two-process run: its blocks of a 2 x 2 split on cuda:0, strips through gloo."""
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        sys.path.insert(0, root)
        from datetime import timedelta
        import torch
        import torch.distributed as dist
        import paper_2208_01260_gb300 as hw
        from paper_2208_01260_gb300 import decomp
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=timedelta(seconds=120))
        sc = _scenario(120, 88, S.REFLECTIVE, S.PERIODIC, seed=66)
        g = hw.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y, dim=2)
        params = hw.make_params()
        plan = decomp.Plan(g, 2, 2, ws)
        comm = decomp.Comm.from_torch(timeout_s=60.0)
        blocks = {p: decomp.CudaBlock(g, params, 2, 2, p) for p in plan.local_parts(rank)}
        decomp.initialise(blocks, plan, comm, lambda p: decomp.window12(sc, plan.info[p]))
        for _ in range(5):
            decomp.rk3_step(blocks, plan, comm)
        q.put((rank, {p: b.state() for p, b in blocks.items()}, comm.host_staging))
        for b in blocks.values():
            b.close()
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error: %r" % e, None))


def test_protocol_two_processes_on_the_gpu(hw):
    """The multi-process protocol across two processes, each with its blocks of a 2 x 2 split on this GPU
    (strips and alpha keys through gloo, staged in host memory; the blocks' kernels never wait on one
    another), 5 steps, against the undecomposed solver bit for bit: the cross-rank halo pairing, the
    periodic wrap across ranks and the all-reduced alpha with the library's CUDA blocks."""
    import torch.multiprocessing as mp
    from paper_2208_01260_gb300 import decomp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    procs = [ctx.Process(target=_gpu_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = [q.get(timeout=300) for _ in range(2)]
    finally:
        for p in procs:
            p.join(60)
            if p.exitcode is None:
                p.kill()
    states = {}
    for rank, st, staged in res:
        assert not isinstance(st, str), st
        assert staged
        states.update(st)
    assert sorted(states) == [0, 1, 2, 3]
    sc = _scenario(120, 88, S.REFLECTIVE, S.PERIODIC, seed=66)
    ref = hw.Solver.from_scenario(sc, hw.make_params())
    ref.advance(5, use_graph=False)
    g = hw.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y, dim=2)
    got = decomp.gather(decomp.Plan(g, 2, 2, 2), states)
    for qq, (a, b) in enumerate(zip(ref.state(), got)):
        assert np.array_equal(a, b), (qq, float(np.abs(a - b).max()))
    ref.close()


def _adjoint_problem(hw, sc, nsteps, ng, seed):
    rng = np.random.default_rng(seed)
    ref = hw.Solver.from_scenario(sc, hw.make_params())
    dts = [ref.cfl_dt()] * nsteps
    ref.close()
    gidx = rng.choice(sc.nx * sc.ny, ng, replace=False).astype(np.int32)
    obs = 1.0 + 0.002 * rng.normal(size=nsteps * ng)
    return dts, gidx, obs


def _undecomposed_adjoint(hw, sc, dts, gidx, obs):
    import torch
    from paper_2208_01260_gb300 import adjoint as A
    ref = hw.Solver.from_scenario(sc, hw.make_params())
    gs = torch.empty(9, sc.ny, sc.nx, dtype=torch.float64, device="cuda")
    gb = torch.empty(3, sc.ny, sc.nx, dtype=torch.float64, device="cuda")
    loss, _ = A.hw_adjoint_run(ref.h, dts, gidx, obs, A.HW_ADJ_TAPE, [gs[q] for q in range(9)], [gb[q] for q in range(3)])
    ref.close()
    return loss, gs.cpu().numpy(), gb.cpu().numpy()


def _check_adjoint_grads(plan, grads, ref_s, ref_b):
    scale = float(np.abs(ref_s).max())
    for p, (gs, gb) in grads.items():
        i = plan.info[p]
        win = (slice(i.j0, i.j0 + i.ny), slice(i.i0, i.i0 + i.nx))
        for q in range(9):
            assert np.abs(gs[q] - ref_s[q][win]).max() <= 1e-10 * scale, (p, q)
        for q in range(3):
            assert np.abs(gb[q] - ref_b[q][win]).max() <= 1e-10 * scale, (p, 9 + q)


def test_adjoint_protocol_in_one_process(hw):
    """The multi-process adjoint (decomp.adjoint_run over hw_part_adj_*) with all 2 x 2 blocks in this process
    against the undecomposed adjoint on its whole-run tape: the loss bit for bit, the gradients to 1e-10 of the
    largest state-gradient entry (the alpha adjoint's shares summed in another order)."""
    from paper_2208_01260_gb300 import decomp
    sc = _scenario(96, 66, S.REFLECTIVE, S.PERIODIC, seed=64)
    dts, gidx, obs = _adjoint_problem(hw, sc, 5, 9, 8)
    g = hw.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y, dim=2)
    params = hw.make_params()
    plan = decomp.Plan(g, 2, 2, 1)
    comm = decomp.Comm(0, 1)
    blocks = {p: decomp.CudaBlock(g, params, 2, 2, p) for p in plan.local_parts(0)}
    decomp.initialise(blocks, plan, comm, lambda p: decomp.window12(sc, plan.info[p]))
    loss, grads = decomp.adjoint_run(blocks, plan, comm, dts, gidx, obs)
    for b in blocks.values():
        b.close()
    ref_loss, ref_s, ref_b = _undecomposed_adjoint(hw, sc, dts, gidx, obs)
    assert loss == ref_loss
    _check_adjoint_grads(plan, grads, ref_s, ref_b)


def _gpu_adjoint_rank(rank, ws, port, q):
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        sys.path.insert(0, root)
        from datetime import timedelta
        import torch
        import torch.distributed as dist
        import paper_2208_01260_gb300 as hw
        from paper_2208_01260_gb300 import decomp
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=timedelta(seconds=120))
        sc = _scenario(96, 66, S.PERIODIC, S.REFLECTIVE, seed=67)
        dts, gidx, obs = _adjoint_problem(hw, sc, 4, 8, 9)
        g = hw.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y, dim=2)
        params = hw.make_params()
        plan = decomp.Plan(g, 2, 2, ws)
        comm = decomp.Comm.from_torch(timeout_s=60.0)
        blocks = {p: decomp.CudaBlock(g, params, 2, 2, p) for p in plan.local_parts(rank)}
        decomp.initialise(blocks, plan, comm, lambda p: decomp.window12(sc, plan.info[p]))
        loss, grads = decomp.adjoint_run(blocks, plan, comm, dts, gidx, obs)
        q.put((rank, loss, grads))
        for b in blocks.values():
            b.close()
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error: %r" % e, None))


def test_adjoint_protocol_two_processes_on_the_gpu(hw):
    """The multi-process adjoint across two processes on this GPU (2 x 2 blocks, two per rank; strips, keys,
    gauge values and alpha adjoints through gloo): both ranks find the undecomposed adjoint's loss bit for bit
    and their blocks' gradients within 1e-10 of the largest state-gradient entry, with periodic wrap across
    ranks along x and walls along y."""
    import torch.multiprocessing as mp
    from paper_2208_01260_gb300 import decomp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    procs = [ctx.Process(target=_gpu_adjoint_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = [q.get(timeout=600) for _ in range(2)]
    finally:
        for p in procs:
            p.join(60)
            if p.exitcode is None:
                p.kill()
    for r in res:
        assert not isinstance(r[1], str), r[1]
    sc = _scenario(96, 66, S.PERIODIC, S.REFLECTIVE, seed=67)
    dts, gidx, obs = _adjoint_problem(hw, sc, 4, 8, 9)
    ref_loss, ref_s, ref_b = _undecomposed_adjoint(hw, sc, dts, gidx, obs)
    g = hw.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y, dim=2)
    plan = decomp.Plan(g, 2, 2, 2)
    parts = []
    for rank, loss, grads in res:
        assert loss == ref_loss, (rank, loss, ref_loss)
        _check_adjoint_grads(plan, grads, ref_s, ref_b)
        parts += list(grads)
    assert sorted(parts) == [0, 1, 2, 3]


def test_part_adjoint_argument_and_order_errors(hw):
    """hw_part_adj_*: a gauge off the block's own nodes, step, stage, face, mode and plane-set arguments out
    of range (HW_ERR_ARG), the reverse before hw_part_adj_set_misfit and an alpha application without a
    reverse stage (HW_ERR_STATE); a context on a solver that is not a block is refused."""
    import torch
    from paper_2208_01260_gb300 import decomp
    sc = _scenario(64, 48, S.REFLECTIVE, S.REFLECTIVE, seed=68)
    g = hw.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y, dim=2)
    params = hw.make_params()
    plan = decomp.Plan(g, 2, 1, 1)
    comm = decomp.Comm(0, 1)
    blocks = {p: decomp.CudaBlock(g, params, 2, 1, p) for p in plan.local_parts(0)}
    decomp.initialise(blocks, plan, comm, lambda p: decomp.window12(sc, plan.info[p]))
    blk = blocks[0]
    with pytest.raises(hw.HwError) as e:  # node (40, 5) lies on block 1
        hw.PartAdjoint(blk.h, 2, 1, [0], [5 * sc.nx + 40], sc.nx)
    assert e.value.code == -1
    a = hw.PartAdjoint(blk.h, 2, 1, [0], [5 * sc.nx + 3], sc.nx)
    strip = torch.zeros(a.strip_size(0, hw.HW_FACE_E), dtype=torch.float64, device="cuda")
    keys = torch.zeros(2, dtype=torch.int64, device="cuda")
    for call in (lambda: a.pack(2, 1, hw.HW_FACE_E, strip), lambda: a.pack(0, 4, hw.HW_FACE_E, strip),
                 lambda: a.pack(0, 1, 7, strip), lambda: a.unpack(0, 1, hw.HW_FACE_E, 9, strip),
                 lambda: a.rpack(2, hw.HW_FACE_E, strip), lambda: a.forward_stage(0, 1, -1.0, keys),
                 lambda: a.strip_size(3, hw.HW_FACE_E)):
        with pytest.raises(hw.HwError) as e:
            call()
        assert e.value.code == -1
    with pytest.raises(hw.HwError) as e:
        a.reverse_stage(1, 3, 1e-3)
    assert e.value.code == -6
    a.set_misfit(np.zeros(2), np.zeros(2))
    with pytest.raises(hw.HwError) as e:
        a.alpha_apply([0.0, 0.0], [0, 0])
    assert e.value.code == -6
    a.close()
    s = hw.Solver.from_scenario(sc, params)
    with pytest.raises(hw.HwError) as e:
        hw.PartAdjoint(s.h, 2, 1, [0], [3], sc.nx)
    assert e.value.code == -1
    s.close()
    for b in blocks.values():
        b.close()
