"""The allocation-free 1D right-hand side against the regular entry point.

hw_rhs1d_noalloc serves callers that must not allocate device memory (a memory pool that owns the
GPU, or a time-critical loop that cannot pay for cudaMalloc); it keeps its working memory in a fixed
device array inside the library. This test calls it through the C ABI twice in a row on different
grids (the second call reuses the array the first one left behind), then once more on the first grid,
and checks each result against hw_create + hw_init + hw_rhs on the same inputs with the tolerance of
the other right-hand-side parity tests. It also checks that grids above the limit are rejected.
"""
import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S
from _parity import normwise, rhs_scales

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _regular(hw, sc, params):
    s = hw.Solver.from_scenario(sc, params, device=True)
    import torch
    out = [torch.empty(sc.nx, dtype=torch.float64, device="cuda") for _ in range(4)]
    hw.hw_rhs(s.h, out)
    torch.cuda.synchronize()
    r = [o.cpu().numpy() for o in out]
    s.close()
    return r


def _noalloc(hw, sc, params):
    import torch
    grid = hw.make_grid(sc.nx, 1, sc.x0, sc.x1, bc_x=sc.bc_x, dim=1)
    out = [torch.full((sc.nx,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(4)]
    hw.hw_rhs1d_noalloc(grid, params, _dev(sc.h), _dev(sc.hu), _dev(sc.b), [_dev(d) for d in sc.deriv], out)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in out]


def _scales(orc, sc):
    st, stat = orc.to_state1d(sc.h, sc.hu, sc.b, sc.deriv)
    return rhs_scales(st, stat, sc.dx)


def test_noalloc_matches_regular_entry_point(orc):
    import torch
    import paper_2208_01260_gb300 as hw
    assert torch.cuda.is_available()
    a = S.perturbed1d(perturb=0.05)
    b = S.accuracy1d(3000)
    pa = hw.make_params(eps_w=a.eps_w)
    pb = hw.make_params(eps_w=b.eps_w)
    ref_a = _regular(hw, a, pa)
    ref_b = _regular(hw, b, pb)
    first = _noalloc(hw, a, pa)
    second = _noalloc(hw, b, pb)
    third = _noalloc(hw, a, pa)
    for got, ref, sc in [(first, ref_a, a), (second, ref_b, b), (third, ref_a, a)]:
        assert all(np.all(np.isfinite(x)) for x in got)
        err = normwise(got, ref, _scales(orc, sc))
        assert max(err) <= 1e-12, err


def test_noalloc_rejects_grids_above_the_limit():
    import torch
    import paper_2208_01260_gb300 as hw
    n = 16385
    grid = hw.make_grid(n, 1, 0.0, 1.0, dim=1)
    z = [torch.ones(n, dtype=torch.float64, device="cuda") for _ in range(10)]
    with pytest.raises(hw.HwError) as e:
        hw.hw_rhs1d_noalloc(grid, hw.make_params(), z[0], z[1], z[2], z[3:6], z[6:10])
    assert e.value.code == -1 and "HW_NOALLOC_MAX_NX" in str(e.value)
