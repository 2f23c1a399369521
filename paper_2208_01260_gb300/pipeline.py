"""Streams of independent jobs through the public API: each job uploads a state from host memory, advances
it by a number of SSP-RK3 steps (Sec. 2.2 eq. RK, CFL time steps on the device) and downloads the result.

Jobs are dealt round-robin to `lanes` solvers of the same grid, each with its own CUDA stream and its own
host thread, so that one job's uploads and downloads run while another job's steps occupy the GPU (the
library's calls release the interpreter while they run and wait only on their own solver's stream).
Within a lane the jobs run one after the other, each as `set_state`, `advance`, `get_state`.
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
