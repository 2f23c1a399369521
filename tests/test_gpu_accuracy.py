"""Fifth-order convergence of the CUDA path on the paper's accuracy tests (Ex. 4.1 in 1D to t = 0.1,
Ex. 4.6 in 2D to t = 0.05; smooth periodic data), by self-refinement with dt ~ dx^(5/3) so that the
third-order time error is O(dx^5): the error between grids N and 2N at the shared nodes falls by about
32 per refinement."""
import math

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


def _run(hw, sc, t_end, n0):
    s = hw.Solver.from_scenario(sc, hw.make_params())
    dx = sc.dx
    t = 0.0
    while t < t_end - 1e-14:
        a = s.alpha()
        rate = a[0] / sc.dx + (a[1] / sc.dy if sc.dim == 2 else 0.0)
        dt = 0.6 / rate * (dx * n0) ** (2.0 / 3.0)
        dt = min(dt, t_end - t)
        s.rk3_step(dt)
        t += dt
    out = s.state()
    s.close()
    return out


def test_fifth_order_1d_ex41(hw):
    res = {n: _run(hw, S.accuracy1d(n), 0.1, 50) for n in (200, 400, 800)}
    sub = slice(None, None, 2)
    orders = [math.log2(np.abs(res[200][q] - res[400][q][sub]).mean() /
                        np.abs(res[400][q] - res[800][q][sub]).mean()) for q in range(2)]
    assert min(orders) > 4.6, orders


def test_fifth_order_2d_ex46(hw):
    res = {n: _run(hw, S.ex46(n), 0.05, 40) for n in (40, 80, 160)}
    sub = (slice(None, None, 2), slice(None, None, 2))
    orders = [math.log2(np.abs(res[40][q] - res[80][q][sub]).mean() /
                        np.abs(res[80][q] - res[160][q][sub]).mean()) for q in range(3)]
    assert min(orders) > 4.5, orders
