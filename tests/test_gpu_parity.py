"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Sizes span several tiles of every kernel (x-sweep 189 interfaces per row tile, y-sweep 32 columns per
block, node 32x8) with ragged tails; the full-size 2048^2 workload is checked on sampled nodes the
oracle computes one by one. See tests/_parity.py for the tolerances.
"""

import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S
from _parity import (normwise, oracle_grid, oracle_state, rel_l1, rhs_scales, stage_scales, tiny_derivatives)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hw():
    import paper_2208_01260_gb300 as hw
    import torch
    assert torch.cuda.is_available()
    hw.lib()
    return hw


def solver(hw, sc, **pk):
    params = hw.make_params(eps_w=pk.pop("eps_w", sc.eps_w), **pk)
    return hw.Solver.from_scenario(sc, params)


def oparams(orc, sc, **pk):
    return orc.make_params(eps_w=pk.pop("eps_w", sc.eps_w), **pk)


CASES_2D = [
    ("hump_reflective", lambda: S.hump2d(70, 45, seed=21), {}),
    ("hump_periodic", lambda: S.hump2d(131, 67, seed=22, bc=S.PERIODIC), {}),
    ("strip_reflective", lambda: S.bumps2d(150, 80, strip=0.01), {}),
    ("ex46_periodic", lambda: S.ex46(48), {}),
    ("no_char", lambda: S.hump2d(40, 37, seed=23), {"char_decomp": 0}),
    ("linear", lambda: S.hump2d(40, 37, seed=24), {"linear_weights": 1}),
    ("tiny_eps", lambda: S.bumps2d(66, 33, strip=1e-3), {"eps_w": 1e-10}),
    ("min_grid", lambda: S.hump2d(2, 3, seed=25), {}),
    ("three_x_tiles", lambda: S.hump2d(450, 40, seed=26), {}),
    ("int_mul_fallback", lambda: tiny_derivatives(S.hump2d(70, 45, seed=27)), {}),
]


@pytest.mark.parametrize("name,make,pk", CASES_2D, ids=[c[0] for c in CASES_2D])
def test_rhs_parity_2d(hw, orc, name, make, pk):
    sc = make()
    s = solver(hw, sc, **dict(pk))
    R = s.rhs()
    st, stat = oracle_state(orc, sc)
    Ro, al = orc.rhs2d(oracle_grid(orc, sc), oparams(orc, sc, **dict(pk)), st, stat)
    a = s.alpha()
    assert abs(a[0] - al[0]) <= 1e-14 * al[0] and abs(a[1] - al[1]) <= 1e-14 * al[1]
    err = normwise(R, Ro, rhs_scales(st, stat, min(sc.dx, sc.dy)))
    assert max(err) <= 1e-12, err


@pytest.mark.parametrize("name,make,pk", CASES_2D, ids=[c[0] for c in CASES_2D])
def test_stage_parity_2d(hw, orc, name, make, pk):
    """Each of the three stages from identical inputs (the GPU's previous stage and base)."""
    sc = make()
    s = solver(hw, sc, **dict(pk))
    g, p = oracle_grid(orc, sc), oparams(orc, sc, **dict(pk))
    st, stat = oracle_state(orc, sc)
    dt = orc.cfl_dt2d(g, p, st, stat)
    assert abs(s.cfl_dt() - dt) <= 1e-14 * dt
    cur = s.state()
    base = None
    for k in (1, 2, 3):
        s.rk3_stage(k, dt)
        out_gpu = s.state()
        out_orc, base_orc, _ = orc.stage2d(g, p, k, dt, cur, stat, base)
        err = normwise(out_gpu, out_orc, stage_scales(cur, stat))
        assert max(err) <= 1e-12, (k, err)
        if k == 1:
            base_gpu = s.base()
            errb = normwise(base_gpu, base_orc, stage_scales(cur, stat))
            assert max(errb) <= 1e-12, errb
            base = base_gpu
        cur = out_gpu


@pytest.mark.parametrize("name,make,pk,tol", [
    ("hump_reflective", lambda: S.hump2d(64, 48, seed=31), {}, 1e-9),
    ("strip_reflective", lambda: S.bumps2d(96, 48, strip=0.01), {}, 1e-8),
    ("ex46_periodic", lambda: S.ex46(32), {}, 1e-9),
])
def test_multistep_parity_2d(hw, orc, name, make, pk, tol):
    sc = make()
    s = solver(hw, sc, **pk)
    g, p = oracle_grid(orc, sc), oparams(orc, sc, **pk)
    st, stat = oracle_state(orc, sc)
    cur = st
    for _ in range(12):
        dt = orc.cfl_dt2d(g, p, cur, stat)
        cur = orc.rk3_step2d(g, p, dt, cur, stat)
        s.rk3_step(dt)
    err = rel_l1(s.state(), cur)
    assert max(err) <= tol, err


def test_lake_at_rest_gpu(hw):
    sc = S.bumps2d(256, 128, strip=0.0)
    s = solver(hw, sc)
    t, n = s.advance(200)
    assert n == 200
    out = s.state()
    res = max(np.abs(out[0] - 1.0).max(), np.abs(out[1]).max(), np.abs(out[2]).max())
    assert res <= 1e-12, res


def test_lake_at_rest_gpu_2048(hw):
    """The benchmark's 2048^2 reflective bathymetry without the perturbation strip, 200 RK3 steps."""
    sc = S.bumps2d(2048, 2048, strip=0.0)
    s = solver(hw, sc)
    t, n = s.advance(200)
    out = s.state()
    res = max(np.abs(out[0] - 1.0).max(), np.abs(out[1]).max(), np.abs(out[2]).max())
    assert res <= 1e-12, res


def test_final_time_parity_2048(hw, orc):
    """The benchmark workload at full size (2048^2, reflective, 8 bumps + 0.01 strip): 12 RK3 steps at
    the CFL step, the GPU from its captured graph with the time step found on the device, the oracle with
    its own steps; the simulated times, the normwise error per group, and the relative L1 error per group:
    U and V at the discontinuous-data bound (1e-8). The strip varies in x only, so the y-derivatives Q
    stay near zero (their L1 norm is about 1e-5 of V's) and their relative L1 error measures conditioning:
    Q is held to ten times the oracle's own change when its input moves by one unit in the last place."""
    sc = S.bumps2d(2048, 2048, strip=0.01)
    s = solver(hw, sc)
    g, p = oracle_grid(orc, sc), oparams(orc, sc)
    st, stat = oracle_state(orc, sc)
    nsteps = 12
    t, n = s.advance(nsteps, use_graph=True)
    assert n == nsteps
    got = s.state()
    s.close()

    def run(state):
        cur, tt = state, 0.0
        for _ in range(nsteps):
            dt = orc.cfl_dt2d(g, p, cur, stat)
            cur = orc.rk3_step2d(g, p, dt, cur, stat)
            tt += dt
        return cur, tt
    cur, tref = run(st)
    assert abs(t - tref) <= 1e-13 * tref, (t, tref)
    err = rel_l1(got, cur)
    assert max(err[:2]) <= 1e-8, err
    assert max(normwise(got, cur, stage_scales(cur, stat))) <= 1e-11
    # the oracle against itself with eta moved by one ulp at every node (random signs)
    rng = np.random.default_rng(1)
    st2 = [a.copy() for a in st]
    st2[0] = st2[0] * (1.0 + rng.choice([-1.0, 1.0], st2[0].shape) * 2.0 ** -52)
    cur2, _ = run(st2)
    sens = rel_l1(cur2, cur)
    assert err[2] <= 10 * sens[2], (err, sens)


def test_sampled_parity_2048(hw, orc):
    """Full-size workload (2048^2, reflective, 8 bumps + strip), each stage on 3000 sampled nodes."""
    sc = S.bumps2d(2048, 2048, strip=0.01)
    s = solver(hw, sc)
    g, p = oracle_grid(orc, sc), oparams(orc, sc)
    st, stat = oracle_state(orc, sc)
    pi, pj = S.random_sample(2048, 2048, 3000, seed=7)
    dt = s.cfl_dt()
    cur = st
    base_pts = None
    for k in (1, 2, 3):
        al = orc.alpha2d(g, p, cur, stat)
        a = s.alpha()
        assert abs(a[0] - al[0]) <= 1e-14 * al[0]
        s.rk3_stage(k, dt)
        out = s.state()
        o_pts, mod_pts = orc.stage2d_points(g, p, k, dt, cur, stat, al, pi, pj, base_pts)
        gpu_pts = np.stack([out[q][pj, pi] for q in range(9)], axis=1)
        err = normwise([gpu_pts[:, q] for q in range(9)], [o_pts[:, q] for q in range(9)], stage_scales(cur, stat))
        assert max(err) <= 1e-12, (k, err)
        if k == 1:
            b = s.base()
            base_pts = np.stack([b[q][pj, pi] for q in range(9)], axis=1)
        cur = out


# ------------------------------------------------------------------------------------------------
# 1D
# ------------------------------------------------------------------------------------------------
CASES_1D = [
    ("perturbed_small", lambda: S.perturbed1d(), {}),
    ("perturbed_large", lambda: S.perturbed1d(perturb=0.2), {}),
    ("accuracy_periodic", lambda: S.accuracy1d(300), {}),
    ("no_char", lambda: S.perturbed1d(perturb=0.05), {"char_decomp": 0}),
    ("linear", lambda: S.accuracy1d(130), {"linear_weights": 1}),
    ("ex42_step", lambda: S.ex42(200, step=True), {}),
    ("min_grid", lambda: S.accuracy1d(2), {}),
]


@pytest.mark.parametrize("name,make,pk", CASES_1D, ids=[c[0] for c in CASES_1D])
def test_rhs_and_stage_parity_1d(hw, orc, name, make, pk):
    sc = make()
    s = solver(hw, sc, **dict(pk))
    g, p = oracle_grid(orc, sc), oparams(orc, sc, **dict(pk))
    st, stat = oracle_state(orc, sc)
    R = s.rhs()
    Ro, al = orc.rhs1d(g, p, st, stat)
    assert max(normwise(R, Ro, rhs_scales(st, stat, sc.dx))) <= 1e-12
    dt = orc.cfl_dt1d(g, p, st, stat)
    assert abs(s.cfl_dt() - dt) <= 1e-14 * dt
    cur, base = s.state(), None
    for k in (1, 2, 3):
        s.rk3_stage(k, dt)
        out = s.state()
        oo, bo, _ = orc.stage1d(g, p, k, dt, cur, stat, base)
        assert max(normwise(out, oo, stage_scales(cur, stat))) <= 1e-12, k
        if k == 1:
            base = s.base()
        cur = out


def test_config1_final_time(hw, orc):
    """1D N=200 reflective, two bumps, 1e-3 pulse, eps = 1e-10, CFL 0.6 to t = 0.2."""
    sc = S.perturbed1d()
    s = solver(hw, sc)
    g, p = oracle_grid(orc, sc), oparams(orc, sc)
    st, stat = oracle_state(orc, sc)
    out_o, t_o, n_o = orc.run1d(g, p, st, stat, 0.2)
    t, n = s.advance(10 ** 6, t_end=0.2)
    assert n == n_o and abs(t - 0.2) < 1e-14
    err = rel_l1(s.state(), out_o)
    assert max(err) <= 1e-8, err


# ------------------------------------------------------------------------------------------------
# API behaviour
# ------------------------------------------------------------------------------------------------
def test_graph_matches_eager(hw):
    sc = S.hump2d(100, 77, seed=41)
    a = solver(hw, sc)
    b = solver(hw, sc)
    a.advance(6, use_graph=True)
    b.advance(6, use_graph=False)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)


def test_advance_to_end_time(hw):
    sc = S.hump2d(64, 64, seed=42)
    s = solver(hw, sc)
    t, n = s.advance(10 ** 6, t_end=0.05)
    assert abs(t - 0.05) < 1e-14
    x = s.state()
    t2, n2 = s.advance(5, t_end=0.05)
    assert n2 == 0 and t2 == 0.0
    for a, b in zip(x, s.state()):
        assert np.array_equal(a, b)


def test_state_roundtrip_and_device_pointers(hw):
    import torch
    # derivative planes are stored times the grid spacing: the round trip is exact when the spacing is
    # a power of two, and within one rounding of the scaling otherwise
    for nx, ny, exact in [(64, 32, True), (64, 48, False)]:
        sc = S.hump2d(nx, ny, seed=43)
        s = solver(hw, sc)
        s.rk3_step(s.cfl_dt())
        x = s.state()
        s.set_state(x)
        for a, b in zip(x, s.state()):
            if exact:
                assert np.array_equal(a, b)
            else:
                assert np.all(np.abs(a - b) <= 4.5e-16 * np.abs(a))
    sc = S.hump2d(64, 48, seed=43)
    # device-pointer init and rhs give the same numbers as the host path
    d = hw.Solver.from_scenario(sc, hw.make_params(), device=True)
    h = hw.Solver.from_scenario(sc, hw.make_params(), device=False)
    outs = [torch.empty(sc.ny, sc.nx, dtype=torch.float64, device="cuda") for _ in range(9)]
    hw.hw_rhs(d.h, outs)
    torch.cuda.synchronize()
    for a, b in zip(outs, h.rhs()):
        assert np.array_equal(a.cpu().numpy(), b)


def test_errors(hw):
    sc = S.hump2d(16, 16, seed=44)
    with pytest.raises(hw.HwError) as e:
        hw.Solver(hw.make_grid(1, 16, dim=2), hw.make_params())
    assert e.value.code == -1
    s = hw.Solver(hw.make_grid(16, 16, 0, 1, 0, 1, 1, 1), hw.make_params())
    with pytest.raises(hw.HwError) as e:
        s.rk3_step(1e-3)
    assert e.value.code == -6
    bad = sc.h.copy()
    bad[3, 4] = -0.1
    with pytest.raises(hw.HwError) as e:
        hw.hw_init(s.h, bad, sc.hu, sc.hv, sc.b, sc.deriv)
    assert e.value.code == -2
    bad[3, 4] = np.nan
    with pytest.raises(hw.HwError) as e:
        hw.hw_init(s.h, bad, sc.hu, sc.hv, sc.b, sc.deriv)
    assert e.value.code == -3
    # a NaN velocity is found by the next alpha reduction
    hw.hw_init(s.h, sc.h, sc.hu, sc.hv, sc.b, sc.deriv)
    hu = sc.hu.copy()
    hu[5, 5] = np.inf
    st = s.state(hw.HW_LAYOUT_PHYSICAL)
    st[1] = hu
    hw.hw_set_state(s.h, st, hw.HW_LAYOUT_PHYSICAL)
    with pytest.raises(hw.HwError) as e:
        s.alpha()
    assert e.value.code == -3


def test_checkpoint_and_resume_is_bitwise(hw):
    """Checkpoint (state in the equilibrium layout, time, step count) after 7 steps, restore into a fresh
    solver, continue: equal bit for bit to the uninterrupted run (grid spacing 2^-6, so the derivative
    scalings are exact; the physical layout's h = eta - b would round)."""
    sc = S.hump2d(64, 64, seed=47)
    a = solver(hw, sc)
    a.advance(7, use_graph=False)
    st = a.state(hw.HW_LAYOUT_EQUILIBRIUM)
    t, n = hw.hw_get_time(a.h)
    assert n == 7 and t > 0
    a.advance(5, t_end=10.0, use_graph=False)
    b = solver(hw, sc)
    hw.hw_set_state(b.h, st, hw.HW_LAYOUT_EQUILIBRIUM)
    hw.hw_set_time(b.h, t, n)
    b.advance(5, t_end=10.0, use_graph=False)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)
    assert hw.hw_get_time(a.h) == hw.hw_get_time(b.h)


def test_time_and_state_api_errors(hw):
    sc = S.hump2d(32, 32, seed=48)
    s = solver(hw, sc)
    L = hw.lib()
    with pytest.raises(hw.HwError) as e:
        hw.hw_set_time(s.h, -1.0, 0)
    assert e.value.code == -1
    with pytest.raises(hw.HwError) as e:
        hw.hw_set_time(s.h, 0.0, -5)
    assert e.value.code == -1
    assert L.hw_get_time(s.h.ptr, None, None) == -1
    # a resumed float solver keeps its time too
    s32 = hw.Solver.from_scenario(sc, hw.make_params(precision=hw.HW_FP32))
    s32.advance(3, use_graph=False)
    t, n = hw.hw_get_time(s32.h)
    assert n == 3 and t > 0
    base = s32.base()
    assert len(base) == 9 and np.isfinite(base[0]).all()
