"""The allocation-free 1D right-hand side against the regular entry point.

hw_rhs1d_noalloc serves callers that must not allocate device memory (a memory pool that owns the
GPU, or a time-critical loop that cannot pay for cudaMalloc); it keeps its working memory in a fixed
device array inside the library. This test calls it through the C ABI twice in a row on different
grids (the second call reuses the array the first one left behind), then once more on the first grid,
and checks each result against hw_create + hw_init + hw_rhs on the same inputs with the tolerance of
the other right-hand-side parity tests; it does the same at exactly the largest grid the array holds.
It also checks that grids above the limit are rejected, and that a depth error is reported by the
call that received the bad input and not by the next valid call.
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


def test_noalloc_at_the_largest_grid(orc):
    """nx = HW_NOALLOC_MAX_NX fills the array up to its last interface plane and its counters."""
    import paper_2208_01260_gb300 as hw
    sc = S.accuracy1d(16384)
    p = hw.make_params(eps_w=sc.eps_w)
    ref = _regular(hw, sc, p)
    for _ in range(2):
        got = _noalloc(hw, sc, p)
        assert all(np.all(np.isfinite(x)) for x in got)
        err = normwise(got, ref, _scales(orc, sc))
        assert max(err) <= 1e-12, err


def test_noalloc_reports_bad_depth_once():
    """A host-made input with h <= 0 gives HW_ERR_DEPTH; the next call with valid input returns HW_OK."""
    import dataclasses
    import paper_2208_01260_gb300 as hw
    sc = S.perturbed1d(perturb=0.05)
    p = hw.make_params(eps_w=sc.eps_w)
    h = sc.h.copy()
    h[17] = -0.5
    bad = dataclasses.replace(sc, h=h)
    with pytest.raises(hw.HwError) as e:
        _noalloc(hw, bad, p)
    assert e.value.code == -2
    h = sc.h.copy()
    h[5] = float("nan")
    with pytest.raises(hw.HwError) as e:
        _noalloc(hw, dataclasses.replace(sc, h=h), p)
    assert e.value.code == -3
    got = _noalloc(hw, sc, p)
    assert all(np.all(np.isfinite(x)) for x in got)


def test_noalloc_rejects_grids_above_the_limit():
    import torch
    import paper_2208_01260_gb300 as hw
    n = 16385
    grid = hw.make_grid(n, 1, 0.0, 1.0, dim=1)
    z = [torch.ones(n, dtype=torch.float64, device="cuda") for _ in range(10)]
    with pytest.raises(hw.HwError) as e:
        hw.hw_rhs1d_noalloc(grid, hw.make_params(), z[0], z[1], z[2], z[3:6], z[6:10])
    assert e.value.code == -1 and "HW_NOALLOC_MAX_NX" in str(e.value)
