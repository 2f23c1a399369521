"""The hand-written discrete adjoint against central differences of the CUDA forward map and against
forward-mode dual numbers through the CPU oracle; checkpointing schedules; the autograd Function."""
import functools

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


def _eq_static(sc):
    import torch
    st = [sc.h + sc.b, sc.hu, sc.hv, sc.deriv[0] + sc.deriv[6], sc.deriv[1], sc.deriv[2], sc.deriv[3] + sc.deriv[7],
          sc.deriv[4], sc.deriv[5]]
    stat = [sc.b, sc.deriv[6], sc.deriv[7]]
    T = lambda a: torch.tensor(np.stack(a), dtype=torch.float64, device="cuda").contiguous()
    return T(st), T(stat), [np.array(a) for a in st], [np.array(a) for a in stat]


def _smooth_direction(sc, seed, scale=1.0, static=True):
    """Sums of Gaussians with consistent analytic derivatives (state: eta and its derivatives; static:
    b and its derivatives), plus small momentum perturbations."""
    rng = np.random.default_rng(seed)
    x = S.axis(sc.nx, sc.x0, sc.x1, sc.bc_x)
    y = S.axis(sc.ny, sc.y0, sc.y1, sc.bc_y)
    X, Y = np.meshgrid(x, y)

    def bumps(k):
        f = np.zeros_like(X); fx = np.zeros_like(X); fy = np.zeros_like(X)
        for _ in range(k):
            A, xc, yc, s = rng.normal(), rng.uniform(sc.x0, sc.x1), rng.uniform(sc.y0, sc.y1), rng.uniform(0.1, 0.3)
            g = A * np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / s ** 2)
            f += g; fx += -2 * (X - xc) / s ** 2 * g; fy += -2 * (Y - yc) / s ** 2 * g
        return f, fx, fy
    e, ex, ey = bumps(3)
    m, mx, my = bumps(2)
    w, wx, wy = bumps(2)
    dst = [scale * a for a in (e, 0.1 * m, 0.1 * w, ex, 0.1 * mx, 0.1 * wx, ey, 0.1 * my, 0.1 * wy)]
    if static:
        b, bx, by = bumps(2)
        dstat = [0.1 * scale * a for a in (b, bx, by)]
    else:
        dstat = [np.zeros_like(X)] * 3
    return dst, dstat


def _forward_step(hw, solver, state, static, dt):
    from paper_2208_01260_gb300 import adjoint as A
    import torch
    A.load_problem(solver, state, static)
    solver.rk3_step(dt)
    out = [torch.empty_like(state[0]) for _ in range(9)]
    hw.hw_get_state(solver.h, out, hw.HW_LAYOUT_EQUILIBRIUM)
    torch.cuda.synchronize()
    return torch.stack(out)


def _strip_and_hump():
    """Perturbation strip next to a wall plus a surface hump, so max(|u|+c) is attained at one node
    (alpha = max is not differentiable where several nodes tie)."""
    sc = S.bumps2d(48, 24, strip=0.01)
    x = S.axis(sc.nx, sc.x0, sc.x1, sc.bc_x)
    y = S.axis(sc.ny, sc.y0, sc.y1, sc.bc_y)
    X, Y = np.meshgrid(x, y)
    g = 0.06 * np.exp(-((X - 1.4) ** 2 + (Y - 0.5) ** 2) / 0.1 ** 2)
    sc.h = sc.h + g
    sc.deriv[0] = sc.deriv[0] - 2 * (X - 1.4) / 0.01 * g
    sc.deriv[3] = sc.deriv[3] - 2 * (Y - 0.5) / 0.01 * g
    return sc


CASES = [
    ("hump_reflective", lambda: S.hump2d(40, 33, seed=61, hump_max=0.05), {}),
    ("ex46_periodic", lambda: S.ex46(32), {}),
    ("strip_and_hump", _strip_and_hump, {}),
    ("strip_and_hump_no_limiter", _strip_and_hump, {"limiter": 0}),
    ("no_limiter", lambda: S.hump2d(32, 28, seed=63), {"limiter": 0}),
    ("hump_transmissive", lambda: S.hump2d(40, 33, seed=61, hump_max=0.05, bc=S.OUTFLOW), {}),
]


def _unique_alpha(sc):
    h = sc.h
    c = np.sqrt(9.812 * h)
    for mom in (sc.hu, sc.hv):
        a = np.sort((np.abs(mom / h) + c).ravel())[::-1]
        if (a[0] - a[1]) <= 1e-9 * a[0]:
            return False
    return True


@pytest.mark.parametrize("name,make,pk", CASES, ids=[c[0] for c in CASES])
def test_adjoint_step_dot_product(hw, name, make, pk):
    import torch
    from paper_2208_01260_gb300 import adjoint as A
    sc = make()
    assert _unique_alpha(sc)
    solver = hw.Solver.from_scenario(sc, hw.make_params(**pk))
    state, static, _, _ = _eq_static(sc)
    A.load_problem(solver, state, static)
    dt = solver.cfl_dt()
    rng = np.random.default_rng(7)
    lam = torch.tensor(rng.normal(size=state.shape), dtype=torch.float64, device="cuda")
    dst, dstat = _smooth_direction(sc, 11)
    vs = torch.tensor(np.stack(dst), dtype=torch.float64, device="cuda")
    vb = torch.tensor(np.stack(dstat), dtype=torch.float64, device="cuda")
    # adjoint
    A.load_problem(solver, state, static)
    ls = lam.clone()
    lb = torch.zeros_like(static)
    A.hw_adjoint_step(solver.h, dt, [ls[q] for q in range(9)], [lb[q] for q in range(3)])
    torch.cuda.synchronize()
    adj = float((ls * vs).sum() + (lb * vb).sum())
    # central differences
    eps = 1e-6
    fp = _forward_step(hw, solver, state + eps * vs, static + eps * vb, dt)
    fm = _forward_step(hw, solver, state - eps * vs, static - eps * vb, dt)
    fd = float((lam * (fp - fm)).sum()) / (2 * eps)
    assert abs(adj - fd) <= 1e-6 * abs(fd) + 1e-9, (adj, fd)


def _oracle_problem(sc, nsteps, ng, seed):
    import oracle
    g = oracle.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y)
    p = oracle.make_params()
    st, stat = oracle.to_state2d(sc.h, sc.hu, sc.hv, sc.b, sc.deriv)
    dt = oracle.cfl_dt2d(g, p, st, stat)
    rng = np.random.default_rng(seed)
    gidx = rng.choice(sc.nx * sc.ny, ng, replace=False).astype(np.int32)
    obs = 1.0 + 0.002 * rng.normal(size=nsteps * ng)
    return g, p, st, stat, np.full(nsteps, dt), gidx, obs


def test_adjoint_run_matches_oracle_dual_numbers(hw):
    import torch
    import oracle
    from paper_2208_01260_gb300 import adjoint as A
    sc = S.hump2d(32, 24, seed=71, hump_max=0.05)
    nsteps, ng = 6, 7
    g, p, st, stat, dts, gidx, obs = _oracle_problem(sc, nsteps, ng, 3)
    solver = hw.Solver.from_scenario(sc, hw.make_params())
    state, static, _, _ = _eq_static(sc)
    A.load_problem(solver, state, static)
    gs = torch.empty_like(state)
    gb = torch.empty_like(static)
    loss, nf = A.hw_adjoint_run(solver.h, dts, gidx, obs, 2, [gs[q] for q in range(9)], [gb[q] for q in range(3)])
    for seed in (1, 2, 3):
        dst, dstat = _smooth_direction(sc, seed)
        L, dL = oracle.gauge_loss_dual2d(g, p, st, stat, dst, dstat, dts, gidx, obs)
        assert abs(loss - L) <= 1e-10 * abs(L)
        gv = float((gs.cpu().numpy() * np.stack(dst)).sum() + (gb.cpu().numpy() * np.stack(dstat)).sum())
        assert abs(gv - dL) <= 1e-7 * abs(dL) + 1e-12, (gv, dL)


@pytest.mark.parametrize("bc", [S.REFLECTIVE, S.PERIODIC], ids=["reflective", "periodic"])
def test_adjoint_run_matches_oracle_dual_numbers_multi_tile(hw, bc):
    """A grid spanning three x-tiles of the adjoint x-sweep (61 interfaces each) and several y-segments,
    so that the record adjoints a block shares with its neighbours (added with atomics) meet the oracle's
    forward-mode derivative, on walls and on periodic wrap-around."""
    import torch
    import oracle
    from paper_2208_01260_gb300 import adjoint as A
    sc = S.hump2d(160, 48, seed=72, hump_max=0.05, bc=bc)
    nsteps, ng = 4, 9
    g, p, st, stat, dts, gidx, obs = _oracle_problem(sc, nsteps, ng, 4)
    solver = hw.Solver.from_scenario(sc, hw.make_params())
    state, static, _, _ = _eq_static(sc)
    A.load_problem(solver, state, static)
    gs = torch.empty_like(state)
    gb = torch.empty_like(static)
    loss, nf = A.hw_adjoint_run(solver.h, dts, gidx, obs, A.HW_ADJ_TAPE, [gs[q] for q in range(9)],
                                [gb[q] for q in range(3)])
    for seed in (4, 5):
        dst, dstat = _smooth_direction(sc, seed)
        L, dL = oracle.gauge_loss_dual2d(g, p, st, stat, dst, dstat, dts, gidx, obs)
        assert abs(loss - L) <= 1e-10 * abs(L)
        gv = float((gs.cpu().numpy() * np.stack(dst)).sum() + (gb.cpu().numpy() * np.stack(dstat)).sum())
        assert abs(gv - dL) <= 1e-7 * abs(dL) + 1e-12, (gv, dL)
    solver.close()


@functools.lru_cache(None)
def _dp_cost(n, s):
    if n == 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    return min(m + _dp_cost(n - m, s - 1) + _dp_cost(m, s) for m in range(1, n))


def test_checkpointing_schedules_agree(hw):
    import torch
    from paper_2208_01260_gb300 import adjoint as A
    sc = S.hump2d(24, 20, seed=81)
    nsteps, ng = 9, 4
    _, _, _, _, dts, gidx, obs = _oracle_problem(sc, nsteps, ng, 5)
    solver = hw.Solver.from_scenario(sc, hw.make_params())
    state, static, _, _ = _eq_static(sc)
    def current():
        now = [torch.empty_like(state[0]) for _ in range(9)]
        hw.hw_get_state(solver.h, now, hw.HW_LAYOUT_EQUILIBRIUM)
        torch.cuda.synchronize()
        return torch.stack(now)
    grads = []
    for snaps in (0, 1, 3, nsteps - 1, A.HW_ADJ_TAPE, A.HW_ADJ_AUTO):
        A.load_problem(solver, state, static)
        start = current()
        gs = torch.empty_like(state)
        gb = torch.empty_like(static)
        loss, nf = A.hw_adjoint_run(solver.h, dts, gidx, obs, snaps, [gs[q] for q in range(9)], [gb[q] for q in range(3)])
        # the tape (chosen by AUTO on a grid this small) recomputes nothing
        assert nf == (nsteps if snaps < 0 else nsteps + _dp_cost(nsteps, snaps))
        grads.append((gs.cpu().numpy(), gb.cpu().numpy()))
        assert torch.equal(current(), start)  # the solver is back at the initial state
    for gs, gb in grads[1:]:
        # equal up to the summation order of the atomic scatters
        np.testing.assert_allclose(gs, grads[0][0], rtol=1e-9, atol=1e-10 * np.abs(grads[0][0]).max())
        np.testing.assert_allclose(gb, grads[0][1], rtol=1e-9, atol=1e-10 * np.abs(grads[0][1]).max())


def test_autograd_function(hw):
    import torch
    from paper_2208_01260_gb300 import adjoint as A
    sc = S.hump2d(28, 26, seed=91)
    nsteps, ng = 5, 6
    _, _, _, _, dts, gidx, obs = _oracle_problem(sc, nsteps, ng, 9)
    solver = hw.Solver.from_scenario(sc, hw.make_params())
    state, static, _, _ = _eq_static(sc)
    s_ = state.clone().requires_grad_(True)
    b_ = static.clone().requires_grad_(True)
    L = A.GaugeMisfit.apply(s_, b_, solver, dts, gidx, obs)
    L.backward()
    A.load_problem(solver, state, static)
    gs = torch.empty_like(state)
    gb = torch.empty_like(static)
    loss, _ = A.hw_adjoint_run(solver.h, dts, gidx, obs, 2, [gs[q] for q in range(9)], [gb[q] for q in range(3)])
    assert abs(float(L.detach()) - loss) <= 1e-14 * loss
    np.testing.assert_allclose(s_.grad.cpu().numpy(), gs.cpu().numpy(), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(b_.grad.cpu().numpy(), gb.cpu().numpy(), rtol=1e-10, atol=1e-14)


def test_adjoint_gradient_central_differences_20_directions(hw):
    """The adjoint workload (bottom of the benchmark plus a surface hump, reflective, 32 gauges,
    observations from a run with another hump) at 256^2 over 60 steps with the unperturbed CFL step
    sequence: gradient against central differences (step 1e-6) along 20 random smooth directions."""
    import torch
    from paper_2208_01260_gb300 import adjoint as A
    n, nsteps = 256, 60
    sc = S.adjoint_case(n)
    obs_sc = S.adjoint_case(n, hump_seed=1)
    gidx = S.gauges(sc.nx, sc.ny)
    solver = hw.Solver.from_scenario(sc, hw.make_params())
    state, static, _, _ = _eq_static(sc)
    A.load_problem(solver, state, static)
    dts = []
    for _ in range(nsteps):
        dt = solver.cfl_dt()
        dts.append(dt)
        solver.rk3_step(dt)
    obs_solver = hw.Solver.from_scenario(obs_sc, hw.make_params())
    ostate, ostatic, _, _ = _eq_static(obs_sc)
    A.load_problem(obs_solver, ostate, ostatic)
    _, gv = A.hw_gauge_loss(obs_solver.h, dts, gidx, np.zeros(nsteps * len(gidx)))
    obs = gv.ravel()
    A.load_problem(solver, state, static)
    gs = torch.empty_like(state)
    gb = torch.empty_like(static)
    loss, nf = A.hw_adjoint_run(solver.h, dts, gidx, obs, 8, [gs[q] for q in range(9)], [gb[q] for q in range(3)])
    G_s, G_b = gs.cpu().numpy(), gb.cpu().numpy()
    eps = 1e-6
    ads, fds = [], []
    for k in range(20):
        dst, dstat = _smooth_direction(sc, 1000 + k, scale=1.0, static=(k % 2 == 0))
        vs = torch.tensor(np.stack(dst), dtype=torch.float64, device="cuda")
        vb = torch.tensor(np.stack(dstat), dtype=torch.float64, device="cuda")
        A.load_problem(solver, state + eps * vs, static + eps * vb)
        lp, _ = A.hw_gauge_loss(solver.h, dts, gidx, obs)
        A.load_problem(solver, state - eps * vs, static - eps * vb)
        lm, _ = A.hw_gauge_loss(solver.h, dts, gidx, obs)
        fds.append((lp - lm) / (2 * eps))
        ads.append(float((G_s * np.stack(dst)).sum() + (G_b * np.stack(dstat)).sum()))
    ads, fds = np.array(ads), np.array(fds)
    # The difference quotient's own error (eps^2 truncation, rounding of L over eps) is absolute, on the
    # scale of the loss's sensitivity, so a direction whose derivative nearly cancels (|fd| far below
    # the others) is held to 1e-6 of one thousandth of the largest |fd| rather than of its own.
    floor = 1e-3 * np.abs(fds).max()
    rel = np.abs(ads - fds) / np.maximum(np.abs(fds), floor)
    assert rel.max() <= 1e-6, (rel.max(), int(rel.argmax()), ads, fds)
    assert np.linalg.norm(ads - fds) <= 1e-6 * np.linalg.norm(fds)


def test_adjoint_buffers_follow_the_solver(hw):
    """Working buffers belong to one solver and are freed with it: solvers of different sizes created
    and destroyed in turn (so a new one may reuse an old one's host address) each get a correct step."""
    import torch
    from paper_2208_01260_gb300 import adjoint as A
    for n in (24, 56, 40):
        sc = S.bumps2d(n, n, strip=0.01)
        solver = hw.Solver.from_scenario(sc, hw.make_params())
        state, static, _, _ = _eq_static(sc)
        A.load_problem(solver, state, static)
        dt = solver.cfl_dt()
        lam = [torch.ones_like(state[0]) * 1e-3 for _ in range(9)]
        lst = [torch.zeros_like(state[0]) for _ in range(3)]
        A.hw_adjoint_step(solver.h, dt, lam, lst)
        torch.cuda.synchronize()
        assert all(torch.isfinite(p).all() for p in lam + lst)
        solver.close()


def test_config5_full_size_gradient_against_central_differences(hw):
    """The adjoint workload at its full size: 512^2, 400 steps at the unperturbed CFL dt sequence, 32
    gauges, observations from a run with another hump; the tape-mode gradient against central
    differences (step 1e-6) along 20 random smooth directions, with the scale floor of the 256^2 test."""
    import torch
    from paper_2208_01260_gb300 import adjoint as A
    n, nsteps = 512, 400
    sc = S.adjoint_case(n)
    obs_sc = S.adjoint_case(n, hump_seed=1)
    gidx = S.gauges(sc.nx, sc.ny)
    solver = hw.Solver.from_scenario(sc, hw.make_params())
    state, static, _, _ = _eq_static(sc)
    A.load_problem(solver, state, static)
    dts = []
    for _ in range(nsteps):
        dt = solver.cfl_dt()
        dts.append(dt)
        solver.rk3_step(dt)
    obs_solver = hw.Solver.from_scenario(obs_sc, hw.make_params())
    ostate, ostatic, _, _ = _eq_static(obs_sc)
    A.load_problem(obs_solver, ostate, ostatic)
    _, gv = A.hw_gauge_loss(obs_solver.h, dts, gidx, np.zeros(nsteps * len(gidx)))
    obs_solver.close()
    obs = gv.ravel()
    A.load_problem(solver, state, static)
    gs = torch.empty_like(state)
    gb = torch.empty_like(static)
    loss, nf = A.hw_adjoint_run(solver.h, dts, gidx, obs, A.HW_ADJ_AUTO, [gs[q] for q in range(9)],
                                [gb[q] for q in range(3)])
    assert nf == nsteps  # the tape fits: nothing recomputed
    G_s, G_b = gs.cpu().numpy(), gb.cpu().numpy()
    eps = 1e-6
    ads, fds = [], []
    for k in range(20):
        dst, dstat = _smooth_direction(sc, 2000 + k, scale=1.0, static=(k % 2 == 0))
        vs = torch.tensor(np.stack(dst), dtype=torch.float64, device="cuda")
        vb = torch.tensor(np.stack(dstat), dtype=torch.float64, device="cuda")
        A.load_problem(solver, state + eps * vs, static + eps * vb)
        lp, _ = A.hw_gauge_loss(solver.h, dts, gidx, obs)
        A.load_problem(solver, state - eps * vs, static - eps * vb)
        lm, _ = A.hw_gauge_loss(solver.h, dts, gidx, obs)
        fds.append((lp - lm) / (2 * eps))
        ads.append(float((G_s * np.stack(dst)).sum() + (G_b * np.stack(dstat)).sum()))
    ads, fds = np.array(ads), np.array(fds)
    floor = 1e-3 * np.abs(fds).max()
    rel = np.abs(ads - fds) / np.maximum(np.abs(fds), floor)
    assert rel.max() <= 1e-6, (rel.max(), int(rel.argmax()), ads, fds)
    assert np.linalg.norm(ads - fds) <= 1e-6 * np.linalg.norm(fds)
    solver.close()
