"""Independent jobs through pipeline.JobPipeline (two solvers on their own streams and host threads) and
pipeline.StagedPipeline (one solver, its copies on an upload and a download stream through two device
staging sets each way) give, job by job, the bits of one solver running the same jobs one after the other."""
import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["two_solvers", "staged"])
def test_pipeline_jobs_equal_serial_jobs(form):
    import torch
    import paper_2208_01260_gb300 as hw
    from paper_2208_01260_gb300.pipeline import JobPipeline, StagedPipeline
    assert torch.cuda.is_available()
    sc = S.hump2d(160, 96, seed=81)
    src = hw.Solver.from_scenario(sc, hw.make_params())
    inputs = []
    for _ in range(5):  # five different states of one run
        src.advance(3, use_graph=False)
        st = src.state(hw.HW_LAYOUT_PHYSICAL)
        inputs.append([torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in st])
    src.close()
    outs = [[torch.empty(sc.ny, sc.nx, dtype=torch.float64).pin_memory().numpy() for _ in range(9)] for _ in inputs]
    pipe = JobPipeline(sc, hw.make_params(), lanes=2) if form == "two_solvers" else StagedPipeline(sc, hw.make_params())
    pipe.run(inputs, outs, nsteps=2)
    pipe.run(inputs[:1], outs[:1], nsteps=2)  # a second run reuses the staging sets
    pipe.close()
    ref = hw.Solver.from_scenario(sc, hw.make_params())
    for i, planes in enumerate(inputs):
        hw.hw_set_state(ref.h, planes, hw.HW_LAYOUT_PHYSICAL)
        ref.advance(2, use_graph=False)
        want = ref.state(hw.HW_LAYOUT_PHYSICAL)
        for q in range(9):
            assert np.array_equal(outs[i][q], want[q]), (i, q)
    ref.close()
