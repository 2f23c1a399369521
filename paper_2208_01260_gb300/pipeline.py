"""Streams of independent jobs through the public API: each job uploads a state from host memory, advances
it by a number of SSP-RK3 steps (Sec. 2.2 eq. RK, CFL time steps on the device) and downloads the result.

JobPipeline deals the jobs round-robin to `lanes` solvers of the same grid, each with its own CUDA stream
and its own host thread, so that one job's uploads and downloads run while another job's steps occupy
the GPU (the library's calls release the interpreter while they run and wait only on their own solver's
stream); the lanes' steps also run side by side. Within a lane the jobs run one after the other, each as
`set_state`, `advance`, `get_state`.

StagedPipeline keeps one solver, so the GPU steps one job at a time: a job's planes go up on an upload
stream into one of two device staging sets while the previous job steps, and its result comes down on a
download stream from one of two output sets while the next job steps (events order the three streams).
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor
from typing import Optional, Sequence

from . import HW_LAYOUT_PHYSICAL, Solver, hw_get_state, hw_params, hw_set_state


class JobPipeline:
    """`lanes` solvers initialised from scenario `sc` (its bottom and grid serve every job)."""

    def __init__(self, sc, params: Optional[hw_params] = None, lanes: int = 2):
        import torch
        if lanes < 1:
            raise ValueError("lanes must be >= 1")
        self.streams = [torch.cuda.Stream() for _ in range(lanes)]
        self.solvers = [Solver.from_scenario(sc, params, stream=s.cuda_stream) for s in self.streams]
        self.pool = ThreadPoolExecutor(max_workers=lanes)

    @property
    def lanes(self) -> int:
        return len(self.solvers)

    def run(self, inputs: Sequence[Sequence], outputs: Sequence[Sequence], nsteps: int = 1,
            layout: int = HW_LAYOUT_PHYSICAL):
        """Job i: the 9 host planes inputs[i] in, nsteps steps, the 9 planes into outputs[i] (pinned host
        memory lets the copies run at the link's rate). Job i runs on lane i % lanes."""
        if len(inputs) != len(outputs):
            raise ValueError("one output per input")

        def lane(k):
            s = self.solvers[k]
            for i in range(k, len(inputs), self.lanes):
                hw_set_state(s.h, inputs[i], layout)
                s.advance(nsteps, use_graph=False)
                hw_get_state(s.h, outputs[i], layout)

        for f in [self.pool.submit(lane, k) for k in range(self.lanes)]:
            f.result()

    def close(self):
        self.pool.shutdown(wait=True)
        for s in self.solvers:
            s.close()
        self.solvers = []


class StagedPipeline:
    """One solver initialised from scenario `sc` (its bottom and grid serve every job), its own compute
    stream, an upload and a download stream, and two device staging sets each way."""

    def __init__(self, sc, params: Optional[hw_params] = None):
        import torch
        self.compute, self.up, self.down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        self.solver = Solver.from_scenario(sc, params, stream=self.compute.cuda_stream)
        n, shape = self.solver.h.nstate, self.solver.shape
        self.stage_in = [[torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(n)] for _ in range(2)]
        self.stage_out = [[torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(n)] for _ in range(2)]

    def run(self, inputs: Sequence[Sequence], outputs: Sequence[Sequence], nsteps: int = 1,
            layout: int = HW_LAYOUT_PHYSICAL):
        """Job i: the host planes inputs[i] in, nsteps steps, the planes into outputs[i] (pinned host memory
        lets the copies run asynchronously at the link's rate). Returns when every result is on the host."""
        import torch
        if len(inputs) != len(outputs):
            raise ValueError("one output per input")
        njobs = len(inputs)
        in_free = [None, None]   # per staging set: the set_state that last read it
        out_free = [None, None]  # per output set: the download that last read it
        ready = []

        def upload(i):
            b = i % 2
            ev = torch.cuda.Event()
            with torch.cuda.stream(self.up):
                if in_free[b] is not None:
                    self.up.wait_event(in_free[b])
                for q, a in enumerate(inputs[i]):
                    self.stage_in[b][q].copy_(torch.from_numpy(a), non_blocking=True)
                ev.record(self.up)
            ready.append(ev)

        if njobs:
            upload(0)
        for i in range(njobs):
            b = i % 2
            if i + 1 < njobs:
                upload(i + 1)  # runs while job i steps
            self.compute.wait_event(ready[i])
            hw_set_state(self.solver.h, self.stage_in[b], layout)  # device planes: ordered on the compute stream
            in_free[b] = torch.cuda.Event()
            in_free[b].record(self.compute)
            if out_free[b] is not None:
                self.compute.wait_event(out_free[b])
            self.solver.advance(nsteps, use_graph=False)
            hw_get_state(self.solver.h, self.stage_out[b], layout)
            done = torch.cuda.Event()
            done.record(self.compute)
            with torch.cuda.stream(self.down):  # runs while job i + 1 steps
                self.down.wait_event(done)
                for q, dst in enumerate(outputs[i]):
                    torch.from_numpy(dst).copy_(self.stage_out[b][q], non_blocking=True)
                out_free[b] = torch.cuda.Event()
                out_free[b].record(self.down)
        self.down.synchronize()
        self.up.synchronize()

    def close(self):
        if self.solver is not None:
            self.compute.synchronize()
            self.solver.close()
            self.solver = None
