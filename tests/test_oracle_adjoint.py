"""Pins of the oracle's forward-mode dual numbers (the reference the GPU adjoint is checked against):
the dual run's loss equals the plain double run's, its directional derivative matches central
differences of the plain double run, and it is linear in the direction."""
import numpy as np
import pytest

from paper_2208_01260_gb300 import scenarios as S


def _direction(sc, seed):
    """Sums of Gaussians for eta and b with their analytic derivatives, plus small momentum terms
    (state in the oracle's equilibrium layout; static b, b_x, b_y)."""
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(S.axis(sc.nx, sc.x0, sc.x1, sc.bc_x), S.axis(sc.ny, sc.y0, sc.y1, sc.bc_y))

    def bumps(k):
        f = np.zeros_like(X); fx = np.zeros_like(X); fy = np.zeros_like(X)
        for _ in range(k):
            A, xc, yc, s = rng.normal(), rng.uniform(sc.x0, sc.x1), rng.uniform(sc.y0, sc.y1), rng.uniform(0.15, 0.3)
            g = A * np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / s ** 2)
            f += g; fx += -2 * (X - xc) / s ** 2 * g; fy += -2 * (Y - yc) / s ** 2 * g
        return f, fx, fy
    e, ex, ey = bumps(2)
    m, mx, my = bumps(1)
    b, bx, by = bumps(1)
    dst = [e, 0.1 * m, 0.0 * m, ex, 0.1 * mx, 0.0 * mx, ey, 0.1 * my, 0.0 * my]
    dstat = [0.1 * b, 0.1 * bx, 0.1 * by]
    return dst, dstat


def _problem(orc, nsteps=3, ng=6):
    sc = S.hump2d(16, 12, seed=5, hump_max=0.05)
    g = orc.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y)
    p = orc.make_params()
    st, stat = orc.to_state2d(sc.h, sc.hu, sc.hv, sc.b, sc.deriv)
    dt = orc.cfl_dt2d(g, p, st, stat)
    rng = np.random.default_rng(17)
    gidx = rng.choice(sc.nx * sc.ny, ng, replace=False).astype(np.int32)
    obs = 1.0 + 0.002 * rng.normal(size=nsteps * ng)
    return sc, g, p, st, stat, np.full(nsteps, dt), gidx, obs


def _plain_loss(orc, g, p, st, stat, dts, gidx, obs):
    """The misfit from the plain double oracle: rk3_step2d, then eta at the gauges."""
    ng = len(gidx)
    cur = [np.array(a, dtype=np.float64) for a in st]
    L = 0.0
    for j, dt in enumerate(dts):
        cur = orc.rk3_step2d(g, p, dt, cur, stat)
        d = cur[0].ravel()[gidx] - obs[j * ng:(j + 1) * ng]
        L += float((d * d).sum())
    return L


def test_dual_loss_equals_plain_loss(orc):
    sc, g, p, st, stat, dts, gidx, obs = _problem(orc)
    dst, dstat = _direction(sc, 1)
    L, _ = orc.gauge_loss_dual2d(g, p, st, stat, dst, dstat, dts, gidx, obs)
    assert abs(L - _plain_loss(orc, g, p, st, stat, dts, gidx, obs)) <= 1e-13 * L


def test_dual_derivative_matches_central_differences(orc):
    sc, g, p, st, stat, dts, gidx, obs = _problem(orc)
    eps = 1e-6
    for seed in (1, 2, 3):
        dst, dstat = _direction(sc, seed)
        _, dL = orc.gauge_loss_dual2d(g, p, st, stat, dst, dstat, dts, gidx, obs)
        plus = _plain_loss(orc, g, p, [a + eps * v for a, v in zip(st, dst)],
                           [a + eps * v for a, v in zip(stat, dstat)], dts, gidx, obs)
        minus = _plain_loss(orc, g, p, [a - eps * v for a, v in zip(st, dst)],
                            [a - eps * v for a, v in zip(stat, dstat)], dts, gidx, obs)
        fd = (plus - minus) / (2 * eps)
        assert abs(dL - fd) <= 1e-6 * abs(fd) + 1e-12, (seed, dL, fd)


def test_dual_derivative_is_linear_in_the_direction(orc):
    sc, g, p, st, stat, dts, gidx, obs = _problem(orc)
    d1, s1 = _direction(sc, 1)
    d2, s2 = _direction(sc, 2)
    _, a = orc.gauge_loss_dual2d(g, p, st, stat, d1, s1, dts, gidx, obs)
    _, b = orc.gauge_loss_dual2d(g, p, st, stat, d2, s2, dts, gidx, obs)
    _, c = orc.gauge_loss_dual2d(g, p, st, stat, [2.0 * x + y for x, y in zip(d1, d2)],
                                 [2.0 * x + y for x, y in zip(s1, s2)], dts, gidx, obs)
    assert c == pytest.approx(2.0 * a + b, rel=1e-12, abs=1e-15)
