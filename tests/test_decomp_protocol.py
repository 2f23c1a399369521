"""The block decomposition on the CPU: the partition (host-only C call) and the halo/alpha protocol of
``paper_2208_01260_gb300.decomp`` across gloo ranks, each block advanced by the CPU oracle, against the
oracle's undecomposed run, bit for bit; and the protocol's failure detection (a rank whose block raises, a
rank that leaves without a word, a dropped halo message): every rank ends with DecompFailure within a few
collective timeouts instead of waiting for ever.

The blocks here are test doubles: each holds its block plus the 2-node ring in host arrays, packs and
unpacks strips with numpy by the rules hwswe.h states for hw_halo_pack / hw_halo_unpack, takes alpha from
the oracle over its extended grid and advances its own nodes with the oracle's stage at those nodes. The
protocol under test (the exchange order and pairing across ranks, the ring of the grid's own boundary,
the all-reduce of alpha, the stage sequence) is the library's. The grids have power-of-two spacings, so
the extended grids' spacings equal the global one exactly, as the GPU block solvers impose.
"""
import os
import socket
import sys
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PER, REF, OUT = 0, 1, 2
ODD_X = {1, 3, 5, 7, 10}   # state planes (9) then b, b_x, b_y: odd across x-walls
ODD_Y = {2, 5, 6, 7, 11}


def _grid(hw, nx, ny, bcx, bcy):
    # dx = dy = 1/64: block origins and extents are exact binary fractions
    return hw.make_grid(nx, ny, 0.0, nx / 64.0, 0.0, ny / 64.0, bcx, bcy, dim=2)


def test_plan_needs_a_block_per_rank():
    import paper_2208_01260_gb300 as hw
    from paper_2208_01260_gb300 import decomp
    g = _grid(hw, 64, 32, PER, PER)
    with pytest.raises(ValueError):
        decomp.Plan(g, 1, 2, 3)
    assert decomp.Plan(g, 1, 2, 2).local_parts(1) == [1]


def test_partition_covers_grid_and_pairs_neighbours():
    import paper_2208_01260_gb300 as hw
    for (nx, ny, px, py, bcx, bcy) in [(48, 40, 3, 2, PER, REF), (50, 33, 4, 3, OUT, PER), (9, 4, 2, 2, REF, OUT),
                                       (64, 64, 1, 1, PER, PER)]:
        g = _grid(hw, nx, ny, bcx, bcy)
        cover = np.zeros((ny, nx), dtype=int)
        infos = [hw.hw_dd_partition(g, px, py, p) for p in range(px * py)]
        for p, i in enumerate(infos):
            assert i.nx >= 2 and i.ny >= 2
            cover[i.j0:i.j0 + i.ny, i.i0:i.i0 + i.nx] += 1
            bx, by = p % px, p // px
            for f, (edge, bc) in enumerate([(bx == 0, bcx), (bx == px - 1, bcx), (by == 0, bcy), (by == py - 1, bcy)]):
                if edge and bc != PER:
                    assert i.mode[f] == (hw.HW_HALO_MIRROR if bc == REF else hw.HW_HALO_REPLICATE) and i.nbr[f] == p
                else:
                    q = i.nbr[f]
                    assert i.mode[f] == hw.HW_HALO_NEIGHBOR
                    assert infos[q].nbr[f ^ 1] == p  # the pairing is symmetric
                    # neighbours across x share the rows, across y the columns
                    if f < 2:
                        assert (infos[q].j0, infos[q].ny) == (i.j0, i.ny)
                    else:
                        assert (infos[q].i0, infos[q].nx) == (i.i0, i.nx)
        assert (cover == 1).all()
    with pytest.raises(hw.HwError):
        hw.hw_dd_partition(_grid(hw, 7, 8, PER, PER), 4, 1, 0)  # a block of 1 node
    with pytest.raises(hw.HwError):
        hw.hw_dd_partition(_grid(hw, 8, 8, PER, PER), 2, 2, 4)


class OracleBlock:
    """A block advanced by the CPU oracle (test double of the library's CudaBlock)."""

    def __init__(self, orc, hw, grid, params, px, py, part):
        import torch
        self.torch, self.orc = torch, orc
        self.info = hw.hw_dd_partition(grid, px, py, part)
        i = self.info
        self.nxe, self.nye = i.nx + 4, i.ny + 4
        dx = (grid.x1 - grid.x0) / grid.nx
        dy = (grid.y1 - grid.y0) / grid.ny
        x0 = grid.x0 + (i.i0 - 2) * dx
        y0 = grid.y0 + (i.j0 - 2) * dy
        self.g = orc.make_grid(self.nxe, self.nye, x0, x0 + self.nxe * dx, y0, y0 + self.nye * dy, OUT, OUT)
        assert self.g.x1 - self.g.x0 == self.nxe * dx and (self.g.x1 - self.g.x0) / self.nxe == dx
        self.dx, self.dy = dx, dy
        self.p = params
        jj, ii = np.meshgrid(np.arange(2, i.ny + 2), np.arange(2, i.nx + 2), indexing="ij")
        self.pi, self.pj = ii.ravel().astype(np.int32), jj.ravel().astype(np.int32)
        self.base = None
        self.dt = None

    # planes of a set: 9 state (+ 3 static at initialisation)
    def _planes(self, set_):
        return self.st + (self.stat if set_ == 1 else [])

    def init(self, arrays, ld):
        h, hu, hv, b = arrays[:4]
        deriv = arrays[4:]
        st, stat = self.orc.to_state2d(h, hu, hv, b, deriv)
        i = self.info
        self.st = [np.zeros((self.nye, self.nxe)) for _ in range(9)]
        self.stat = [np.zeros((self.nye, self.nxe)) for _ in range(3)]
        self.st[0][:] = 1.0  # still water on the ring until the exchange
        for a, src in zip(self.st + self.stat, st + stat):
            a[2:2 + i.ny, 2:2 + i.nx] = src

    def finish_init(self):
        pass

    def strip_size(self, set_, face):
        return len(self._planes(set_)) * 2 * (self.info.ny if face < 2 else self.nxe)

    def new_strip(self, n):
        return self.torch.zeros(n, dtype=self.torch.float64)

    def new_keys(self, n):
        return self.torch.zeros((n, 2), dtype=self.torch.int64)

    def _own(self, face, c):
        ny, nx = self.info.ny, self.info.nx
        return {0: (slice(2, 2 + ny), 2 + c), 1: (slice(2, 2 + ny), nx + c),
                2: (2 + c, slice(None)), 3: (ny + c, slice(None))}[face]

    def _ring(self, face, c):
        ny, nx = self.info.ny, self.info.nx
        return {0: (slice(2, 2 + ny), c), 1: (slice(2, 2 + ny), nx + 2 + c),
                2: (c, slice(None)), 3: (ny + 2 + c, slice(None))}[face]

    def pack(self, set_, face, strip):
        rows = [a[self._own(face, c)] for a in self._planes(set_) for c in (0, 1)]
        strip.numpy()[:] = np.concatenate(rows)

    def unpack(self, set_, face, mode, strip):
        planes = self._planes(set_)
        s = strip.numpy().reshape(len(planes), 2, -1)
        odd = ODD_X if face < 2 else ODD_Y
        for q, a in enumerate(planes):
            for c in (0, 1):
                if mode == 0:
                    v = s[q, c]
                elif mode == 1:
                    v = s[q, 1 - c] * (-1.0 if q in odd else 1.0)
                else:
                    v = s[q, 0 if face in (0, 2) else 1]
                a[self._ring(face, c)] = v

    def alpha_keys(self, row):
        a = self.orc.alpha2d(self.g, self.p, self.st, self.stat)
        row.numpy()[:] = np.ascontiguousarray(a).view(np.int64)

    def max_keys(self, rows, out):
        out.numpy()[:] = rows.numpy().max(axis=0)

    def stage(self, k, keys, t_end):
        alpha = keys.numpy().copy().view(np.float64)
        if k == 1:  # the oracle's CFL step (Sec. 4): cfl / (alpha_x / dx + alpha_y / dy)
            self.dt = self.p.cfl / (alpha[0] / self.dx + alpha[1] / self.dy)
        out, mod = self.orc.stage2d_points(self.g, self.p, k, self.dt, self.st, self.stat, alpha, self.pi, self.pj,
                                           self.base)
        if k == 1:
            cur = np.stack([self.st[q][self.pj, self.pi] for q in range(3)], axis=1)
            self.base = np.concatenate([cur, mod], axis=1)
        for q in range(9):
            self.st[q][self.pj, self.pi] = out[:, q]

    def own_state(self):
        i = self.info
        return [a[2:2 + i.ny, 2:2 + i.nx].copy() for a in self.st]


def _case(name):
    from paper_2208_01260_gb300 import scenarios as S
    import paper_2208_01260_gb300 as hw
    cfg = {"refl_per": (48, 40, REF, PER, 2, 2), "per_out": (48, 36, PER, OUT, 2, 1),
           "out_refl": (40, 48, OUT, REF, 1, 2), "per_per_4": (64, 32, PER, PER, 4, 1)}[name]
    nx, ny, bcx, bcy, px, py = cfg
    sc = S.hump2d(nx, ny, seed=91, box=(0.0, nx / 64.0, 0.0, ny / 64.0), bc=bcx, hump_max=0.05)
    sc.bc_y = bcy
    return sc, _grid(hw, nx, ny, bcx, bcy), px, py


def _rank(rank, ws, port, name, nsteps, q):
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
        sys.path.insert(0, ROOT)
        import torch.distributed as dist
        import oracle as orc
        import paper_2208_01260_gb300 as hw
        from paper_2208_01260_gb300 import decomp
        dist.init_process_group("gloo", rank=rank, world_size=ws)
        sc, grid, px, py = _case(name)
        params = orc.make_params(eps_w=sc.eps_w)
        plan = decomp.Plan(grid, px, py, ws)
        comm = decomp.Comm.from_torch()
        blocks = {p: OracleBlock(orc, hw, grid, params, px, py, p) for p in plan.local_parts(rank)}
        decomp.initialise(blocks, plan, comm, lambda p: decomp.window12(sc, plan.info[p]))
        for _ in range(nsteps):
            decomp.rk3_step(blocks, plan, comm)
        # the undecomposed oracle run (every rank computes it; the grid is small)
        g = orc.make_grid(sc.nx, sc.ny, grid.x0, grid.x1, grid.y0, grid.y1, grid.bc_x, grid.bc_y)
        cur, stat = orc.to_state2d(sc.h, sc.hu, sc.hv, sc.b, sc.deriv)
        for _ in range(nsteps):
            dt = orc.cfl_dt2d(g, params, cur, stat)
            cur = orc.rk3_step2d(g, params, dt, cur, stat)
        bad = []
        for p, blk in blocks.items():
            i = plan.info[p]
            for qq, a in enumerate(blk.own_state()):
                ref = cur[qq][i.j0:i.j0 + i.ny, i.i0:i.i0 + i.nx]
                if not np.array_equal(a, ref):
                    bad.append((p, qq, float(np.abs(a - ref).max())))
        q.put((rank, bad, len(blocks)))
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error: %r" % e, 0))
        raise


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("name", ["refl_per", "per_out", "out_refl", "per_per_4"])
def test_protocol_two_ranks_equals_undecomposed_oracle(name):
    """Two gloo ranks share the blocks (two each for the 2 x 2 and 4 x 1 splits: exchanges within a rank
    and across ranks); after 3 RK3 steps every block's nodes equal the undecomposed oracle run's bitwise,
    for walls, periodic wrap-around (also across ranks) and open boundaries."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, name, 3, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, bad, nb in res:
        assert bad == [], (rank, bad)
        assert nb >= 1


class FailingBlock(OracleBlock):
    """An oracle block whose stage raises at its fail_at-th call (a host-side fault of one block)."""

    def __init__(self, *a, fail_at=None, **k):
        super().__init__(*a, **k)
        self.fail_at, self.nstage = fail_at, 0

    def stage(self, k, keys, t_end):
        self.nstage += 1
        if self.nstage == self.fail_at:
            raise RuntimeError("injected block failure")
        super().stage(k, keys, t_end)


def _dropping_comm(decomp, base, drop_call):
    """A Comm whose drop_call-th exchange leaves out its first send (a message lost on the way)."""
    class Dropping(decomp.Comm):
        calls = 0

        def exchange(self, sends, recvs):
            Dropping.calls += 1
            if Dropping.calls == drop_call and sends:
                sends = sends[1:]
            super().exchange(sends, recvs)
    return Dropping(base.rank, base.world, base.store, base.timeout_s)


def _failing_rank(rank, ws, port, mode, q):
    from datetime import timedelta
    result = None
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
        sys.path.insert(0, ROOT)
        import torch.distributed as dist
        import oracle as orc
        import paper_2208_01260_gb300 as hw
        from paper_2208_01260_gb300 import decomp
        dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=timedelta(seconds=30))
        sc, grid, px, py = _case("refl_per")
        params = orc.make_params(eps_w=sc.eps_w)
        plan = decomp.Plan(grid, px, py, ws)
        comm = decomp.Comm.from_torch(timeout_s=3.0)
        assert comm.store is not None
        if mode == "drop" and rank == 1:
            comm = _dropping_comm(decomp, comm, drop_call=9)  # initialisation x, y; 2 per stage: step 2, stage 1, x faces
        fail_at = 4 if (mode == "raise" and rank == 1) else None  # step 2, stage 1
        blocks = {p: FailingBlock(orc, hw, grid, params, px, py, p, fail_at=fail_at) for p in plan.local_parts(rank)}
        decomp.initialise(blocks, plan, comm, lambda p: decomp.window12(sc, plan.info[p]))
        t0 = time.time()
        try:
            for step in range(4):
                if mode == "leave" and rank == 1 and step == 1:
                    q.put((rank, "left", 0.0))
                    q.close()
                    q.join_thread()
                    os._exit(0)  # gone between steps, nothing reported
                decomp.rk3_step(blocks, plan, comm)
            result = (rank, "completed", time.time() - t0)
        except decomp.DecompFailure as e:
            result = (rank, "DecompFailure: %s" % e, time.time() - t0)
    except Exception as e:  # noqa: BLE001
        result = (rank, "error: %r" % e, 0.0)
    q.put(result)
    q.close()
    q.join_thread()
    os._exit(0)  # leave without tearing down a process group that may have work pending


@pytest.mark.parametrize("mode", ["raise", "leave", "drop"])
def test_protocol_failures_end_every_rank(mode):
    """raise: rank 1's block raises at step 2; rank 1 reports it in the store and raises DecompFailure,
    and rank 0 ends its next collective with DecompFailure naming rank 1's failure. leave: rank 1 exits
    between steps without a word; rank 0's next collective fails within its 3 s bound. drop: rank 1 loses
    one halo message of step 2; rank 0's receive runs out, rank 1's all-reduce runs out or it reads rank
    0's report. No rank runs on, and none waits longer than a few timeouts."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = dict((r, (msg, dt)) for r, msg, dt in (q.get(timeout=120) for _ in range(2)))
    finally:
        for p in procs:
            p.join(30)
            if p.exitcode is None:
                p.kill()
    if mode == "raise":
        assert res[1][0].startswith("DecompFailure: rank 1: block") and "injected block failure" in res[1][0], res
        assert res[0][0].startswith("DecompFailure") and "rank 1: block" in res[0][0], res
    elif mode == "leave":
        assert res[1][0] == "left", res
        assert res[0][0].startswith("DecompFailure: rank 0:"), res
    else:
        assert res[0][0].startswith("DecompFailure: rank 0: halo exchange"), res
        assert res[1][0].startswith("DecompFailure"), res
    for r, (msg, dt) in res.items():
        assert dt < 20.0, (r, msg, dt)


class RingBlock:
    """A numpy block for the exchange and its transpose: 9 extended planes x (forward) and y (adjoint),
    strips packed, unpacked, packed-and-cleared and added by the rules hwswe.h states for hw_halo_pack /
    hw_halo_unpack and hw_part_adj_rpack / hw_part_adj_radd."""

    def __init__(self, info, rng):
        import torch
        self.torch, self.info = torch, info
        self.nxe, self.nye = info.nx + 4, info.ny + 4
        self.x = [np.zeros((self.nye, self.nxe)) for _ in range(9)]
        for a in self.x:
            a[2:-2, 2:-2] = rng.integers(-8, 9, size=(info.ny, info.nx))
        self.y = [rng.integers(-8, 9, size=(self.nye, self.nxe)).astype(np.float64) for _ in range(9)]

    def new_strip(self, n):
        return self.torch.zeros(n, dtype=self.torch.float64)

    def strip_size(self, what, face):
        return 9 * 2 * (self.info.ny if face < 2 else self.nxe)

    def _own(self, face, c):
        ny, nx = self.info.ny, self.info.nx
        return {0: (slice(2, 2 + ny), 2 + c), 1: (slice(2, 2 + ny), nx + c),
                2: (2 + c, slice(None)), 3: (ny + c, slice(None))}[face]

    def _ring(self, face, c):
        ny, nx = self.info.ny, self.info.nx
        return {0: (slice(2, 2 + ny), c), 1: (slice(2, 2 + ny), nx + 2 + c),
                2: (c, slice(None)), 3: (ny + 2 + c, slice(None))}[face]

    @staticmethod
    def _source(face, mode, c):  # the strip offset a ring offset c is copied from
        return c if mode == 0 else (1 - c if mode == 1 else (0 if face in (0, 2) else 1))

    def pack(self, j, k, face, strip):
        strip.numpy()[:] = np.concatenate([a[self._own(face, c)] for a in self.x for c in (0, 1)])

    def unpack(self, j, k, face, mode, strip):
        s = strip.numpy().reshape(9, 2, -1)
        odd = ODD_X if face < 2 else ODD_Y
        for q, a in enumerate(self.x):
            for c in (0, 1):
                v = s[q, self._source(face, mode, c)]
                a[self._ring(face, c)] = -v if (mode == 1 and q in odd) else v

    def rpack(self, what, face, strip):
        strip.numpy()[:] = np.concatenate([a[self._ring(face, c)] for a in self.y for c in (0, 1)])
        for a in self.y:
            for c in (0, 1):
                a[self._ring(face, c)] = 0.0

    def radd(self, what, face, mode, strip):
        s = strip.numpy().reshape(9, 2, -1)
        odd = ODD_X if face < 2 else ODD_Y
        for q, a in enumerate(self.y):
            for c in (0, 1):
                v = s[q, c]
                a[self._own(face, self._source(face, mode, c))] += -v if (mode == 1 and q in odd) else v


def _transpose_rank(rank, ws, port, name, q):
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
        sys.path.insert(0, ROOT)
        import torch
        import torch.distributed as dist
        from paper_2208_01260_gb300 import decomp
        dist.init_process_group("gloo", rank=rank, world_size=ws)
        _, grid, px, py = _case(name)
        plan = decomp.Plan(grid, px, py, ws)
        comm = decomp.Comm.from_torch(timeout_s=30.0)
        blocks = {p: RingBlock(plan.info[p], np.random.default_rng(100 + p)) for p in plan.local_parts(rank)}
        decomp._exchange_stage_input(blocks, plan, comm, 0, 1)  # x: own nodes -> extended (E x)
        lhs = sum(float((a * c).sum()) for b in blocks.values() for a, c in zip(b.x, b.y))  # <E x, y>
        decomp.exchange_adjoint(blocks, plan, comm, 0)  # y -> E^T y on the own nodes, rings cleared
        rhs = sum(float((a[2:-2, 2:-2] * c[2:-2, 2:-2]).sum()) for b in blocks.values() for a, c in zip(b.x, b.y))
        ring_left = sum(float(np.abs(c).sum() - np.abs(c[2:-2, 2:-2]).sum()) for b in blocks.values() for c in b.y)
        t = torch.tensor([lhs, rhs, ring_left], dtype=torch.float64)
        dist.all_reduce(t)
        q.put((rank, t.tolist()))
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error: %r" % e))


@pytest.mark.parametrize("name", ["refl_per", "per_out", "out_refl", "per_per_4"])
def test_adjoint_exchange_is_the_transpose(name):
    """The transposed exchange of the multi-process adjoint (decomp.exchange_adjoint: y faces, then x faces,
    ring strips sent back to the blocks they came from and added there, with the mirror's signs and the
    open end's repeated node) against the forward exchange on two gloo ranks: <E x, y> = <x, E^T y> summed
    over all blocks, exactly (small integers), and every ring left at zero; for walls, periodic wrap across
    ranks, open ends and corners."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_transpose_rank, args=(r, 2, port, name, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, v in res:
        assert not isinstance(v, str), v
        lhs, rhs, rest = v
        assert lhs == rhs and rest == 0.0, (name, lhs, rhs, rest)


def test_batched_instances_partition_across_ranks():
    """The batched form shares its instances among ranks with no communication: every instance on exactly
    one rank, and no rank more than one largest instance above the average load."""
    from paper_2208_01260_gb300 import decomp
    from paper_2208_01260_gb300 import scenarios as S
    nxs, nys = S.batch_sizes(512)
    pts = [int(a) * int(b) for a, b in zip(nxs, nys)]
    for world in (1, 2, 3, 8):
        parts = decomp.partition_instances(pts, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(pts)))
        loads = [sum(pts[i] for i in p) for p in parts]
        assert max(loads) - sum(pts) / world <= max(pts)
    assert decomp.partition_instances([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
