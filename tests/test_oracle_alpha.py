"""Pins of the oracle's Lax-Friedrichs constants (Sec. 2.1 Step 1).

The paper splits the fluxes with a constant alpha and leaves its value unstated; the reading taken
here is the global one, per direction and per RK stage: alpha_x = max over all nodes of the spectral
radius of the flux Jacobian dF1/dU, alpha_y likewise with F2, evaluated on the stage's input state.
For the shallow water equations that radius is |u| + sqrt(g h), which is how the oracle writes it.

These tests reach the same number by another route: the Jacobian of the oracle's pointwise fluxes
(pinned separately against the chain-rule derivative fluxes and the eigen-decomposition) by central
differences at every node, its eigenvalues by numpy, the largest modulus, the maximum over the
nodes. The order and lake-at-rest pins cannot see alpha (its dissipation is O(dx^5) on smooth data
and vanishes at rest), so without these a wrong wave speed, a dropped |u|, a maximum over part of
the grid or an alpha taken from the step's start instead of the stage's input would go unnoticed.
"""
import numpy as np
import pytest

G = 9.812


def _state2d(nx, ny, seed):
    rng = np.random.default_rng(seed)
    b = rng.uniform(-0.2, 0.3, (ny, nx))
    h = rng.uniform(0.3, 2.0, (ny, nx))
    st = [h + b, rng.normal(0.0, 1.0, (ny, nx)), rng.normal(0.0, 1.0, (ny, nx))]
    st += [rng.normal(0.0, 0.3, (ny, nx)) for _ in range(6)]
    stat = [b, rng.normal(0.0, 0.3, (ny, nx)), rng.normal(0.0, 0.3, (ny, nx))]
    return st, stat


def _spectral_radius_max(orc, st, stat, direction, ncomp=3):
    """max over nodes of max |eig(dF/dU)| with dF/dU by central differences of the pointwise flux
    (F1 for direction 0, F2 for direction 1); ncomp = 2 takes the (eta, m) block of F1 (1D)."""
    ny, nx = st[0].shape
    best = 0.0
    for j in range(ny):
        for i in range(nx):
            s12 = np.array([p[j, i] for p in st] + [p[j, i] for p in stat])
            J = np.zeros((ncomp, ncomp))
            for c in range(ncomp):
                d = 1e-6 * max(1.0, abs(s12[c]))
                sp, sm = s12.copy(), s12.copy()
                sp[c] += d
                sm[c] -= d
                J[:, c] = (orc.pointwise2d(G, sp)[direction][:ncomp] - orc.pointwise2d(G, sm)[direction][:ncomp]) / (2 * d)
            best = max(best, float(np.max(np.abs(np.linalg.eigvals(J)))))
    return best


@pytest.mark.parametrize("corner", [False, True])
def test_alpha2d_is_max_spectral_radius(orc, corner):
    nx, ny = 9, 7
    st, stat = _state2d(nx, ny, 11)
    if corner:
        # the largest speeds sit on the boundary (a maximum over interior nodes would miss them)
        st[1][0, 0] = 6.0 * (st[0][0, 0] - stat[0][0, 0])
        st[2][ny - 1, nx - 1] = -7.0 * (st[0][ny - 1, nx - 1] - stat[0][ny - 1, nx - 1])
    g = orc.make_grid(nx, ny, 0.0, 1.0, 0.0, 1.0, orc.BC_REFLECTIVE, orc.BC_REFLECTIVE)
    a = orc.alpha2d(g, orc.make_params(), st, stat)
    ax = _spectral_radius_max(orc, st, stat, 0)
    ay = _spectral_radius_max(orc, st, stat, 1)
    assert abs(a[0] - ax) <= 1e-7 * ax and abs(a[1] - ay) <= 1e-7 * ay, (a, ax, ay)
    if corner:
        assert ax >= 6.0 and ay >= 7.0


def test_alpha2d_follows_the_stage_input(orc):
    """Stages 2 and 3 use alpha of their own input state (the previous stage's output), not of U^n."""
    nx, ny = 8, 6
    st, stat = _state2d(nx, ny, 12)
    g = orc.make_grid(nx, ny, 0.0, 1.0, 0.0, 1.0, orc.BC_PERIODIC, orc.BC_PERIODIC)
    p = orc.make_params()
    dt = orc.cfl_dt2d(g, p, st, stat)
    out1, base, a1 = orc.stage2d(g, p, 1, dt, st, stat)
    out2, _, a2 = orc.stage2d(g, p, 2, dt, out1, stat, base)
    _, _, a3 = orc.stage2d(g, p, 3, dt, out2, stat, base)
    for a, inp in ((a1, st), (a2, out1), (a3, out2)):
        ref = [_spectral_radius_max(orc, inp, stat, d) for d in (0, 1)]
        assert all(abs(a[d] - ref[d]) <= 1e-7 * ref[d] for d in (0, 1)), (a, ref)
    # the stage inputs differ enough that alpha of U^n would fail the check above
    assert max(abs(a2[0] - a1[0]) / a1[0], abs(a3[0] - a1[0]) / a1[0]) > 1e-4
    assert max(abs(a2[1] - a1[1]) / a1[1], abs(a3[1] - a1[1]) / a1[1]) > 1e-4


def test_cfl_dt2d_from_alpha(orc):
    """dt = CFL / (alpha_x/dx + alpha_y/dy) with alpha from the spectral radii (Sec. 4: CFL 0.6)."""
    nx, ny = 6, 5
    st, stat = _state2d(nx, ny, 13)
    g = orc.make_grid(nx, ny, 0.0, 2.0, 0.0, 1.0, orc.BC_REFLECTIVE, orc.BC_PERIODIC)
    dt = orc.cfl_dt2d(g, orc.make_params(), st, stat)
    ax = _spectral_radius_max(orc, st, stat, 0)
    ay = _spectral_radius_max(orc, st, stat, 1)
    ref = 0.6 / (ax / (2.0 / nx) + ay / (1.0 / ny))
    assert abs(dt - ref) <= 1e-7 * ref


def _state1d(n, seed):
    rng = np.random.default_rng(seed)
    b = rng.uniform(-0.2, 0.3, n)
    h = rng.uniform(0.3, 2.0, n)
    return [h + b, rng.normal(0.0, 1.0, n), rng.normal(0.0, 0.3, n), rng.normal(0.0, 0.3, n)], [b, rng.normal(0.0, 0.3, n)]


def _radius1d(orc, st, stat):
    # the 1D flux is the (eta, m) part of F1 with w = 0 and no y-data
    n = len(st[0])
    z = np.zeros((1, n))
    st2 = [st[0][None, :], st[1][None, :], z, st[2][None, :], st[3][None, :], z, z, z, z]
    stat2 = [stat[0][None, :], stat[1][None, :], z]
    return _spectral_radius_max(orc, st2, stat2, 0, ncomp=2)


def test_alpha1d_is_max_spectral_radius_and_follows_the_stage_input(orc):
    n = 16
    st, stat = _state1d(n, 14)
    st[1][n - 1] = 5.0 * (st[0][n - 1] - stat[0][n - 1])  # the fastest node is the last one
    g = orc.make_grid(n, 1, 0.0, 1.0, bc_x=orc.BC_REFLECTIVE)
    p = orc.make_params()
    a0 = orc.alpha1d(g, p, st, stat)
    ref0 = _radius1d(orc, st, stat)
    assert abs(a0 - ref0) <= 1e-7 * ref0 and ref0 >= 5.0
    dt = orc.cfl_dt1d(g, p, st, stat)
    assert abs(dt - 0.6 * (1.0 / n) / ref0) <= 1e-7 * dt
    out1, base, a1 = orc.stage1d(g, p, 1, dt, st, stat)
    out2, _, a2 = orc.stage1d(g, p, 2, dt, out1, stat, base)
    assert abs(a1 - ref0) <= 1e-7 * ref0
    ref2 = _radius1d(orc, out1, stat)
    assert abs(a2 - ref2) <= 1e-7 * ref2
    assert abs(a2 - a1) > 1e-4 * a1
