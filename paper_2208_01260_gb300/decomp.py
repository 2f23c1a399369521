"""Block decomposition of one 2D grid across processes (one process per GPU, or several blocks per process).

The grid is split into px x py blocks (``hw_dd_partition``); block p belongs to rank ``p % world``. Each
block is a solver on its nodes plus a ring of 2 halo nodes (``hw_part_create``). One SSP-RK3 stage
(Sec. 2.2 eq. RK) of the 2D scheme (Sec. 3) is, on every rank:

  1. the halo exchange of the 9 state planes: x faces, then y faces (whose strips span the ring, so the
     corners follow); a block's face takes the neighbour's strip of the opposite face
     (HW_HALO_NEIGHBOR, periodic included) or its own strip mirrored or repeated (walls, open ends);
  2. each block's alpha keys (max(|u|+c), max(|v|+c) over its nodes and ring, as integer bit patterns),
     the maximum over the rank's blocks, then over ranks (one all-reduce of 16 bytes): the global alpha
     of Sec. 2.1 Step 1;
  3. each block's stage with that alpha (stage 1 also takes the CFL step, Sec. 4).

Messages of one exchange phase are posted in one batch, in a global order (receiving block, face) that
every rank follows, so that the i-th message between two ranks is the same on both sides; strips that
stay in the process are unpacked directly. The result equals the undecomposed solver's bit for bit.

The transport is ``torch.distributed`` (NCCL between GPUs, gloo between CPU processes) or nothing for a
single process. Failures are detected on the host, between launches: a rank whose step fails (a block's
error, a collective that failed or outlived ``Comm.timeout_s``) writes the reason under ``ABORT_KEY`` in
the process group's store and raises ``DecompFailure``; every rank reads that key before each stage's
exchange, and its own collectives are bounded by the same timeout, so the others raise ``DecompFailure``
before their next launch or at their next collective instead of waiting for ever. Blocks follow a small interface (``strip_size``, ``new_strip``, ``pack``, ``unpack``,
``alpha_keys``, ``stage``, plus ``max_keys`` of the rank's rows); ``CudaBlock`` is the GPU block of this
library, whose every step runs in its CUDA kernels.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import numpy as np

from . import (HW_FACE_E, HW_FACE_N, HW_FACE_S, HW_FACE_W, HW_HALO_NEIGHBOR, HW_LAYOUT_EQUILIBRIUM, PartAdjoint,
               hw_dd_max_keys, hw_dd_partition, hw_destroy, hw_get_state, hw_grid, hw_halo_pack, hw_halo_strip_size,
               hw_halo_unpack, hw_params, hw_part_alpha_keys, hw_part_create, hw_part_finish_init, hw_part_init,
               hw_part_stage)

ABORT_KEY = "hw_dd_abort"


class DecompFailure(RuntimeError):
    """A rank of the decomposition failed (this one or a peer); the step did not complete."""


FACES_X = (HW_FACE_W, HW_FACE_E)
FACES_Y = (HW_FACE_S, HW_FACE_N)
SET_STATE, SET_INIT = 0, 1


class Plan:
    """Blocks of the grid and their owners."""

    def __init__(self, grid: hw_grid, px: int, py: int, world: int = 1):
        if world < 1 or px * py < world:
            raise ValueError("every rank needs a block: px * py = %d < world = %d" % (px * py, world))
        self.grid, self.px, self.py, self.world = grid, px, py, world
        self.info = [hw_dd_partition(grid, px, py, p) for p in range(px * py)]

    @property
    def nparts(self) -> int:
        return self.px * self.py

    def owner(self, part: int) -> int:
        return part % self.world

    def local_parts(self, rank: int) -> List[int]:
        return [p for p in range(self.nparts) if self.owner(p) == rank]

    def messages(self, faces) -> List[tuple]:
        """(receiving block, its face, sending block) of every NEIGHBOR face in a phase, in the global order."""
        out = []
        for p in range(self.nparts):
            for f in faces:
                if self.info[p].mode[f] == HW_HALO_NEIGHBOR:
                    out.append((p, f, self.info[p].nbr[f]))
        return out


class Comm:
    """Rank, world size, the two collectives the protocol needs (torch.distributed when world > 1), each wait
    bounded by timeout_s, and the failure flag in the store (store: a torch.distributed Store, or None)."""

    def __init__(self, rank: int = 0, world: int = 1, store=None, timeout_s: Optional[float] = None,
                 host_staging: bool = False):
        self.rank, self.world, self.store, self.timeout_s = rank, world, store, timeout_s
        self.host_staging = host_staging  # CUDA tensors travel through host copies (gloo between GPU ranks)

    @classmethod
    def from_torch(cls, timeout_s: Optional[float] = None):
        """The default process group's rank, size and store (None when the group keeps its store private)."""
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            store = None
            try:
                from torch.distributed.distributed_c10d import _get_default_store
                store = _get_default_store()
            except Exception:  # noqa: BLE001
                store = None
            return cls(dist.get_rank(), dist.get_world_size(), store, timeout_s,
                       host_staging=dist.get_backend() == "gloo")
        return cls(0, 1)

    def _wait(self, work, what):
        from datetime import timedelta
        try:
            if self.timeout_s is None:
                work.wait()
            else:
                work.wait(timedelta(seconds=self.timeout_s))
        except Exception as e:  # noqa: BLE001
            raise self.fail("%s: %s: %s" % (what, type(e).__name__, e)) from e

    def exchange(self, sends, recvs):
        """sends: [(tensor, dst_rank, tag)], recvs: [(tensor, src_rank, tag)], both in the global order."""
        if not sends and not recvs:
            return
        import torch.distributed as dist
        staged = []
        if self.host_staging:
            sends = [(t.cpu() if t.is_cuda else t, r, tag) for t, r, tag in sends]
            host_recvs = []
            for t, r, tag in recvs:
                if t.is_cuda:
                    h = t.new_empty(t.shape, device="cpu")
                    staged.append((t, h))
                    t = h
                host_recvs.append((t, r, tag))
            recvs = host_recvs
        # one batch per phase, posted in the global message order (each message is a send or a receive here;
        # the tag is its position in that order, for transports that match by tag)
        merged = [(tag, dist.isend, t, r) for t, r, tag in sends] + [(tag, dist.irecv, t, r) for t, r, tag in recvs]
        merged.sort(key=lambda x: x[0])
        ops = [dist.P2POp(op, t, peer, tag=tag) for tag, op, t, peer in merged]
        try:
            works = dist.batch_isend_irecv(ops)
        except Exception as e:  # noqa: BLE001
            raise self.fail("halo exchange: %s: %s" % (type(e).__name__, e)) from e
        for w in works:
            self._wait(w, "halo exchange")
        for dev, host in staged:
            dev.copy_(host)

    def allreduce(self, t, op: str, what: str):
        """All-reduce of tensor t in place across ranks (op: "max", "min" or "sum"; what names it in errors)."""
        if self.world == 1:
            return
        import torch.distributed as dist
        rop = {"max": dist.ReduceOp.MAX, "min": dist.ReduceOp.MIN, "sum": dist.ReduceOp.SUM}[op]
        buf = t.cpu() if (self.host_staging and t.is_cuda) else t
        try:
            work = dist.all_reduce(buf, op=rop, async_op=True)
        except Exception as e:  # noqa: BLE001
            raise self.fail("%s: %s: %s" % (what, type(e).__name__, e)) from e
        self._wait(work, what)
        if buf is not t:
            t.copy_(buf)

    def allreduce_max(self, t):
        if self.world > 1:
            import torch.distributed as dist
            buf = t.cpu() if (self.host_staging and t.is_cuda) else t
            try:
                work = dist.all_reduce(buf, op=dist.ReduceOp.MAX, async_op=True)
            except Exception as e:  # noqa: BLE001
                raise self.fail("alpha all-reduce: %s: %s" % (type(e).__name__, e)) from e
            self._wait(work, "alpha all-reduce")
            if buf is not t:
                t.copy_(buf)

    def check_peers(self):
        """Raise DecompFailure if any rank has reported a failure (a read of the store, no wait)."""
        if self.store is None or self.world == 1:
            return
        try:
            if self.store.check([ABORT_KEY]):
                raise DecompFailure(self.store.get(ABORT_KEY).decode())
        except DecompFailure:
            raise
        except Exception as e:  # noqa: BLE001  (the store itself is gone: its host rank ended)
            raise DecompFailure("rank %d: store unreachable: %s" % (self.rank, e)) from e

    def fail(self, why: str) -> DecompFailure:
        """Report this rank's failure in the store (first report kept) and return the exception to raise."""
        msg = "rank %d: %s" % (self.rank, why)
        if self.store is not None and self.world > 1:
            try:
                self.store.compare_set(ABORT_KEY, "", msg)
                first = self.store.get(ABORT_KEY).decode()
                if first != msg:
                    msg = "%s (first failure reported: %s)" % (msg, first)
            except Exception:  # noqa: BLE001
                pass
        return DecompFailure(msg)


def exchange(blocks: Dict[int, object], plan: Plan, set_: int, comm: Comm):
    """One halo exchange of plane set `set_` for the rank's blocks (dict part -> block)."""
    for faces in (FACES_X, FACES_Y):
        packed = {}
        for p, blk in blocks.items():
            for f in faces:
                buf = blk.new_strip(blk.strip_size(set_, f))
                blk.pack(set_, f, buf)
                packed[(p, f)] = buf
        sends, recvs, received = [], [], {}
        for order, (p, f, q) in enumerate(plan.messages(faces)):
            mine_p, mine_q = plan.owner(p) == comm.rank, plan.owner(q) == comm.rank
            if mine_q and not mine_p:
                sends.append((packed[(q, f ^ 1)], plan.owner(p), order))
            elif mine_p and not mine_q:
                buf = blocks[p].new_strip(blocks[p].strip_size(set_, f))
                recvs.append((buf, plan.owner(q), order))
                received[(p, f)] = buf
        comm.exchange(sends, recvs)
        for p, blk in blocks.items():
            for f in faces:
                mode = plan.info[p].mode[f]
                if mode == HW_HALO_NEIGHBOR:
                    q = plan.info[p].nbr[f]
                    src = received[(p, f)] if (p, f) in received else packed[(q, f ^ 1)]
                else:
                    src = packed[(p, f)]
                blk.unpack(set_, f, mode, src)


def global_keys(blocks: Dict[int, object], comm: Comm):
    """The alpha keys of the rank's blocks, their maximum, then the maximum over ranks."""
    items = sorted(blocks.items())
    first = items[0][1]
    rows = first.new_keys(len(items))
    for r, (_, blk) in enumerate(items):
        blk.alpha_keys(rows[r])
    keys = first.new_keys(1)[0]
    first.max_keys(rows, keys)
    comm.allreduce_max(keys)
    return keys


def rk3_step(blocks: Dict[int, object], plan: Plan, comm: Comm, t_end: float = -1.0):
    """One SSP-RK3 step of every block of the rank, dt = the CFL step at the step's start. Raises
    DecompFailure (after reporting it) if a block's stage fails here or a peer has reported a failure."""
    for k in (1, 2, 3):
        comm.check_peers()
        exchange(blocks, plan, SET_STATE, comm)
        keys = global_keys(blocks, comm)
        for p, blk in sorted(blocks.items()):
            try:
                blk.stage(k, keys, t_end)
            except DecompFailure:
                raise
            except Exception as e:  # noqa: BLE001
                raise comm.fail("block %d, stage %d: %s: %s" % (p, k, type(e).__name__, e)) from e


def initialise(blocks: Dict[int, object], plan: Plan, comm: Comm, planes12_of):
    """Load every block's own nodes (planes12_of(part) -> (12 arrays, ld)), exchange the state and static
    planes once, then form the b-only source terms."""
    for p, blk in sorted(blocks.items()):
        arrays, ld = planes12_of(p)
        blk.init(arrays, ld)
    exchange(blocks, plan, SET_INIT, comm)
    for _, blk in sorted(blocks.items()):
        blk.finish_init()


class CudaBlock:
    """One block on this process's GPU (the library's block solver); strips and keys are CUDA tensors."""

    def __init__(self, grid: hw_grid, params: hw_params, px: int, py: int, part: int, stream=None):
        import torch
        self.torch = torch
        self.part = part
        self.h = hw_part_create(grid, params, px, py, part, stream)
        self.info = self.h.info
        self.stream = stream

    def close(self):
        hw_destroy(self.h)

    def init(self, planes12: Sequence, ld: int):
        hw_part_init(self.h, planes12, ld)

    def finish_init(self):
        hw_part_finish_init(self.h)

    def strip_size(self, set_: int, face: int) -> int:
        return hw_halo_strip_size(self.h, set_, face)

    def new_strip(self, n: int):
        return self.torch.empty(n, dtype=self.torch.float64, device="cuda")

    def new_keys(self, n: int):
        return self.torch.zeros((n, 2), dtype=self.torch.int64, device="cuda")

    def pack(self, set_: int, face: int, strip):
        hw_halo_pack(self.h, set_, face, strip)

    def unpack(self, set_: int, face: int, mode: int, strip):
        hw_halo_unpack(self.h, set_, face, mode, strip)

    def alpha_keys(self, row):
        hw_part_alpha_keys(self.h, row)

    def max_keys(self, rows, out):
        hw_dd_max_keys(rows, out, self.stream)

    def stage(self, k: int, keys, t_end: float = -1.0):
        hw_part_stage(self.h, k, keys, t_end)

    def state(self, layout: int = HW_LAYOUT_EQUILIBRIUM) -> List[np.ndarray]:
        """The block's own nodes (9 planes, ny x nx each)."""
        nxe, nye = self.info.nx + 4, self.info.ny + 4
        ext = [np.empty((nye, nxe)) for _ in range(9)]
        hw_get_state(self.h, ext, layout)
        return [a[2:-2, 2:-2].copy() for a in ext]


def window12(sc, info) -> tuple:
    """The block's own nodes of a scenario's 12 input planes (host arrays, rows nx apart)."""
    planes = [sc.h, sc.hu, sc.hv, sc.b] + list(sc.deriv)
    out = [np.ascontiguousarray(a[info.j0:info.j0 + info.ny, info.i0:info.i0 + info.nx], dtype=np.float64)
           for a in planes]
    return out, info.nx


def gather(plan: Plan, states: Dict[int, Sequence[np.ndarray]]) -> List[np.ndarray]:
    """Global planes from the blocks' own nodes (host)."""
    g = plan.grid
    out = [np.empty((g.ny, g.nx)) for _ in range(9)]
    for p, planes in states.items():
        i = plan.info[p]
        for q in range(9):
            out[q][i.j0:i.j0 + i.ny, i.i0:i.i0 + i.nx] = planes[q]
    return out


def partition_instances(points: Sequence[int], world: int) -> List[List[int]]:
    """Instances of the batched form shared among `world` ranks with no communication: the largest first,
    each to the rank with the fewest points so far (ties to the lower rank), so every rank's batch has
    about the same work. Returns the instance indices of each rank, in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(points)), key=lambda i: (-int(points[i]), i)):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(i)
        load[r] += int(points[i])
    return [sorted(x) for x in out]


# ------------------------------------------------------------------------------------------------
# The adjoint over the blocks of several processes (the per-block calls hw_part_adj_* of hwswe.h): the
# forward run recorded on every block's tape with the exchanges and the alpha all-reduce of rk3_step,
# the gauge values summed over the blocks, then every stage reversed: the blocks' alpha-adjoint shares
# summed and their first maximising nodes reduced to the global one (applied once, by its owner), and
# the transposed exchange moving ring adjoints back to the nodes they were copied from, y faces first.
# ------------------------------------------------------------------------------------------------
INT_MAX = 2 ** 31 - 1


def gauges_on(plan: Plan, part: int, gauge_idx: Sequence[int]):
    """(slots, global nodes) of the gauges on block `part`'s own nodes."""
    i, gnx = plan.info[part], plan.grid.nx
    slots, nodes = [], []
    for slot, g in enumerate(gauge_idx):
        gi, gj = int(g) % gnx, int(g) // gnx
        if i.i0 <= gi < i.i0 + i.nx and i.j0 <= gj < i.j0 + i.ny:
            slots.append(slot)
            nodes.append(int(g))
    return slots, nodes


class CudaBlockAdjoint:
    """The per-block adjoint context of a CudaBlock (strips and keys as CUDA tensors)."""

    def __init__(self, block: "CudaBlock", nsteps: int, ngauge: int, slots, nodes, global_nx: int):
        self.block = block
        self.a = PartAdjoint(block.h, nsteps, ngauge, slots, nodes, global_nx)

    def close(self):
        self.a.close()

    def new_strip(self, n):
        return self.block.new_strip(n)

    def new_keys(self, n):
        return self.block.new_keys(n)

    def max_keys(self, rows, out):
        self.block.max_keys(rows, out)

    def __getattr__(self, name):  # strip_size, pack, unpack, alpha_keys, forward_stage, ... of PartAdjoint
        return getattr(self.a, name)


def _exchange_stage_input(ctxs, plan: Plan, comm: Comm, j: int, k: int):
    """The forward exchange of the tapes' stage-k inputs of step j (as exchange(), plane set of 9)."""
    for faces in (FACES_X, FACES_Y):
        packed = {}
        for p, c in ctxs.items():
            for f in faces:
                buf = c.new_strip(c.strip_size(0, f))
                c.pack(j, k, f, buf)
                packed[(p, f)] = buf
        sends, recvs, received = [], [], {}
        for order, (p, f, q) in enumerate(plan.messages(faces)):
            mine_p, mine_q = plan.owner(p) == comm.rank, plan.owner(q) == comm.rank
            if mine_q and not mine_p:
                sends.append((packed[(q, f ^ 1)], plan.owner(p), order))
            elif mine_p and not mine_q:
                buf = ctxs[p].new_strip(ctxs[p].strip_size(0, f))
                recvs.append((buf, plan.owner(q), order))
                received[(p, f)] = buf
        comm.exchange(sends, recvs)
        for p, c in ctxs.items():
            for f in faces:
                mode = plan.info[p].mode[f]
                if mode == HW_HALO_NEIGHBOR:
                    q = plan.info[p].nbr[f]
                    src = received[(p, f)] if (p, f) in received else packed[(q, f ^ 1)]
                else:
                    src = packed[(p, f)]
                c.unpack(j, k, f, mode, src)


def exchange_adjoint(ctxs, plan: Plan, comm: Comm, what: int):
    """The transpose of one exchange on the adjoint planes `what` (0: state, 1: static): y faces, then x
    faces; each block's ring strip of a face (cleared) is added to the nodes it was copied from."""
    for faces in (FACES_Y, FACES_X):
        packed = {}
        for p, c in ctxs.items():
            for f in faces:
                buf = c.new_strip(c.strip_size(what, f))
                c.rpack(what, f, buf)
                packed[(p, f)] = buf
        # the forward message (p receives face f from q) runs backwards: p's ring strip goes to q
        sends, recvs, received = [], [], {}
        for order, (p, f, q) in enumerate(plan.messages(faces)):
            mine_p, mine_q = plan.owner(p) == comm.rank, plan.owner(q) == comm.rank
            if mine_p and not mine_q:
                sends.append((packed[(p, f)], plan.owner(q), order))
            elif mine_q and not mine_p:
                buf = ctxs[q].new_strip(ctxs[q].strip_size(what, f ^ 1))
                recvs.append((buf, plan.owner(p), order))
                received[(p, f)] = buf
        comm.exchange(sends, recvs)
        for p, c in sorted(ctxs.items()):
            for f in faces:
                mode = plan.info[p].mode[f]
                if mode != HW_HALO_NEIGHBOR:
                    c.radd(what, f, mode, packed[(p, f)])
                elif plan.owner(plan.info[p].nbr[f]) == comm.rank:
                    ctxs[plan.info[p].nbr[f]].radd(what, f ^ 1, mode, packed[(p, f)])
        for (p, f), buf in sorted(received.items()):
            ctxs[plan.info[p].nbr[f]].radd(what, f ^ 1, HW_HALO_NEIGHBOR, buf)


def _stage_keys(ctxs, comm: Comm, j: int, k: int):
    items = sorted(ctxs.items())
    first = items[0][1]
    rows = first.new_keys(len(items))
    for r, (_, c) in enumerate(items):
        c.alpha_keys(j, k, rows[r])
    keys = first.new_keys(1)[0]
    first.max_keys(rows, keys)
    comm.allreduce_max(keys)
    return keys


def adjoint_run(blocks: Dict[int, object], plan: Plan, comm: Comm, dts: Sequence[float], gauge_idx: Sequence[int],
                eta_obs, make_ctx=None):
    """Gauge misfit sum_j sum_g (eta_g - obs)^2 of a run of len(dts) steps from the blocks' current states and
    its gradient, as hw_dd_adjoint_run but with the blocks spread over ranks. Returns (loss, {part: (9 state
    gradient planes, 3 static ones)}) for the rank's blocks (own nodes, physical units). make_ctx(part, block,
    nsteps, ngauge, slots, nodes, global_nx) builds a block's context (default: CudaBlockAdjoint)."""
    import torch
    nsteps, ngauge = len(dts), len(gauge_idx)
    obs = np.ascontiguousarray(eta_obs, dtype=np.float64).reshape(nsteps * ngauge)
    make_ctx = make_ctx or (lambda p, b, n, ng, sl, nd, gnx: CudaBlockAdjoint(b, n, ng, sl, nd, gnx))
    ctxs = {}
    for p, b in sorted(blocks.items()):
        slots, nodes = gauges_on(plan, p, gauge_idx)
        ctxs[p] = make_ctx(p, b, nsteps, ngauge, slots, nodes, plan.grid.nx)
    try:
        for j in range(nsteps):
            for k in (1, 2, 3):
                comm.check_peers()
                _exchange_stage_input(ctxs, plan, comm, j, k)
                keys = _stage_keys(ctxs, comm, j, k)
                for _, c in sorted(ctxs.items()):
                    c.forward_stage(j, k, dts[j], keys)
        gv = torch.zeros(nsteps * ngauge, dtype=torch.float64)
        for _, c in sorted(ctxs.items()):
            gv += torch.from_numpy(c.gauges())  # each slot is one block's value, zeros elsewhere: exact
        comm.allreduce(gv, "sum", "gauge values")
        g = gv.numpy()
        loss = None
        for _, c in sorted(ctxs.items()):
            loss = c.set_misfit(g, obs)  # the library sums the misfit as its other adjoint entry points do
        for j in reversed(range(nsteps)):
            for k in (3, 2, 1):
                comm.check_peers()
                la = torch.zeros(2, dtype=torch.float64)
                am = torch.full((2,), INT_MAX, dtype=torch.int64)
                for _, c in sorted(ctxs.items()):
                    l, a = c.reverse_stage(j, k, dts[j])
                    la += torch.tensor(l, dtype=torch.float64)
                    am = torch.minimum(am, torch.tensor(a, dtype=torch.int64))
                comm.allreduce(la, "sum", "alpha adjoint")
                comm.allreduce(am, "min", "alpha node")
                for _, c in sorted(ctxs.items()):
                    c.alpha_apply(la.tolist(), am.tolist())
                exchange_adjoint(ctxs, plan, comm, 0)
        for _, c in sorted(ctxs.items()):
            c.finish_static()
        exchange_adjoint(ctxs, plan, comm, 1)
        grads = {p: c.gradients() for p, c in sorted(ctxs.items())}
    except DecompFailure:
        raise
    except Exception as e:  # noqa: BLE001
        raise comm.fail("adjoint: %s: %s" % (type(e).__name__, e)) from e
    finally:
        for c in ctxs.values():
            if hasattr(c, "close"):
                c.close()
    return loss, grads
