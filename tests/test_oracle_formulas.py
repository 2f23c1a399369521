"""Pins of the oracle's scalar building blocks against independent constructions.

Every check here builds its expected value WITHOUT the paper's printed formulas: polynomial data
and exact cell averages, Hermite polynomials obtained by a numpy linear solve, integrals of their
derivatives, finite differences of the flux. A mistyped coefficient, a wrong sign or a swapped
index in the oracle fails one of them.
"""
import numpy as np
import pytest
from numpy.polynomial import Polynomial as P

pytestmark = []


def cell_avgs(poly, centres, dx):
    """Cell averages of poly and of poly' over [c - dx/2, c + dx/2]."""
    I = poly.integ()
    f = np.array([(I(c + dx / 2) - I(c - dx / 2)) / dx for c in centres])
    phi = np.array([(poly(c + dx / 2) - poly(c - dx / 2)) / dx for c in centres])
    return f, phi


def rand_poly(rng, deg, scale=1.0):
    return P(rng.normal(size=deg + 1) * scale)


@pytest.mark.parametrize("seed", range(6))
def test_candidates_exact_for_cubics(orc, seed):
    # Sec. 2.1 eq. (HWEp1): each q_l reproduces a cubic from its cell averages and derivative averages.
    rng = np.random.default_rng(seed)
    dx = rng.uniform(0.01, 0.5)
    xi = rng.uniform(-1, 1)
    poly = rand_poly(rng, 3)
    f, phi = cell_avgs(poly, [xi - dx, xi, xi + dx], dx)
    q = orc.candidates(f, phi, dx)
    np.testing.assert_allclose(q, poly(xi + dx / 2) * np.ones(3), rtol=0, atol=1e-12 * max(1, abs(poly(xi + dx / 2))))
    # and NOT for a generic quartic (the check has teeth)
    poly4 = rand_poly(rng, 4) + P([0, 0, 0, 0, 1.0])
    f4, phi4 = cell_avgs(poly4, [xi - dx, xi, xi + dx], dx)
    q4 = orc.candidates(f4, phi4, dx)
    assert np.max(np.abs(q4 - poly4(xi + dx / 2))) > 1e-9 * dx ** 4


@pytest.mark.parametrize("seed", range(6))
def test_linear_weights_reproduce_quintic(orc, seed):
    # The linear weights (3,3,4)/10 combine the candidates into the quintic Q (exact for degree <= 5).
    rng = np.random.default_rng(100 + seed)
    dx = rng.uniform(0.01, 0.5)
    xi = rng.uniform(-1, 1)
    poly = rand_poly(rng, 5)
    f, phi = cell_avgs(poly, [xi - dx, xi, xi + dx], dx)
    v, w = orc.hweno_value(f, phi, dx, linear=True)
    np.testing.assert_allclose(w, [0.3, 0.3, 0.4], rtol=0, atol=0)
    assert abs(v - poly(xi + dx / 2)) <= 1e-11 * max(1.0, np.max(np.abs(poly.coef)))


@pytest.mark.parametrize("seed", range(6))
def test_qprime_exact_for_quintics(orc, seed):
    # eq. (Rec-phi): Q'(x_{i+1/2}) equals P'(x_{i+1/2}) for any quintic P.
    rng = np.random.default_rng(200 + seed)
    dx = rng.uniform(0.01, 0.5)
    xi = rng.uniform(-1, 1)
    poly = rand_poly(rng, 5)
    f, phi = cell_avgs(poly, [xi - dx, xi, xi + dx], dx)
    d = orc.qprime(f, phi, dx)
    ref = poly.deriv()(xi + dx / 2)
    assert abs(d - ref) <= 1e-9 * max(1.0, np.max(np.abs(poly.coef)))


def _hermite_cubic(cells_f, cells_phi, fvals, phivals, dx):
    """Cubic q with prescribed cell averages of q on `cells_f` and of q' on `cells_phi` (numpy solve)."""
    rows, rhs = [], []
    for c, v in zip(cells_f, fvals):
        rows.append([((c + dx / 2) ** (k + 1) - (c - dx / 2) ** (k + 1)) / ((k + 1) * dx) for k in range(4)])
        rhs.append(v)
    for c, v in zip(cells_phi, phivals):
        rows.append([0.0] + [((c + dx / 2) ** k - (c - dx / 2) ** k) / dx for k in range(1, 4)])
        rhs.append(v)
    return P(np.linalg.solve(np.array(rows), np.array(rhs)))


def _jiang_shu(poly, dx, order):
    """sum_{a=1..order} dx^(2a-1) * integral over [-dx/2, dx/2] of (poly^(a))^2."""
    tot = 0.0
    for a in range(1, order + 1):
        d = poly.deriv(a)
        I = (d * d).integ()
        tot += dx ** (2 * a - 1) * (I(dx / 2) - I(-dx / 2))
    return tot


@pytest.mark.parametrize("seed", range(8))
def test_smoothness_indicators_match_integral_definition(orc, seed):
    # The printed beta_1..beta_3 equal the Jiang-Shu measure of q_1..q_3 on the target cell.
    rng = np.random.default_rng(300 + seed)
    dx = rng.uniform(0.05, 1.0)
    f = rng.normal(size=3)
    phi = rng.normal(size=3)
    q1 = _hermite_cubic([-dx, 0.0], [-dx, 0.0], f[:2], phi[:2], dx)
    q2 = _hermite_cubic([0.0, dx], [0.0, dx], f[1:], phi[1:], dx)
    q3 = _hermite_cubic([-dx, 0.0, dx], [0.0], f, phi[1:2], dx)
    ref = [_jiang_shu(q, dx, 3) for q in (q1, q2, q3)]
    got = orc.smoothness(f, phi, dx)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)
    # the candidate values themselves, from the solved polynomials
    np.testing.assert_allclose(orc.candidates(f, phi, dx), [q(dx / 2) for q in (q1, q2, q3)], rtol=1e-11, atol=1e-12)


def test_weights_properties(orc):
    # eq. (GHYZZ): weights sum to one; smooth data give ~linear weights; a jump kills the crossing stencils.
    dx = 0.01
    x = np.array([-dx, 0, dx])
    f = 1.0 + 0.1 * x
    phi = 0.1 * np.ones(3)
    v, w = orc.hweno_value(f, phi, dx, eps=1e-6)
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(w, [0.3, 0.3, 0.4], atol=1e-6)
    fj = np.array([0.0, 0.0, 1.0])  # jump between i and i+1
    v, w = orc.hweno_value(fj, np.zeros(3), dx, eps=1e-6)
    assert w[0] > 0.999 and w[1] < 1e-6 and w[2] < 1e-6
    assert abs(w.sum() - 1) < 1e-15


def _hermite_quadratic_point(points, mus, dpoints, nus):
    rows, rhs = [], []
    for x, m in zip(points, mus):
        rows.append([1.0, x, x * x]); rhs.append(m)
    for x, n in zip(dpoints, nus):
        rows.append([0.0, 1.0, 2 * x]); rhs.append(n)
    return P(np.linalg.solve(np.array(rows), np.array(rhs)))


@pytest.mark.parametrize("seed", range(6))
def test_limiter_linear_combination_exact_deg4(orc, seed):
    # eqs. (step1-dxi), (limiter-1d): with the linear weights d = (1,1,2)/4 the limited derivative is
    # exact for point data of quartics.
    rng = np.random.default_rng(400 + seed)
    dx = rng.uniform(0.01, 0.5)
    xi = rng.uniform(-1, 1)
    poly = rand_poly(rng, 4)
    xs = np.array([xi - dx, xi, xi + dx])
    mu = poly(xs)
    nu = poly.deriv()(xs)
    v = orc.limiter_value(mu, nu, dx, linear=True)
    assert abs(v - poly.deriv()(xi)) <= 1e-9 * max(1.0, np.max(np.abs(poly.coef)))


@pytest.mark.parametrize("seed", range(6))
def test_limiter_indicators_and_candidates(orc, seed):
    # The printed p'_l(x_i) and beta^L_l follow from the Hermite quadratics p_1..p_3 (numpy solve) and the
    # Jiang-Shu measure on [x_i - dx/2, x_i + dx/2] (first and second derivatives).
    rng = np.random.default_rng(500 + seed)
    dx = rng.uniform(0.05, 1.0)
    mu = rng.normal(size=3)
    nu = rng.normal(size=3)
    p1 = _hermite_quadratic_point([-dx, 0.0], mu[:2], [-dx], nu[:1])
    p2 = _hermite_quadratic_point([0.0, dx], mu[1:], [dx], nu[2:])
    p3 = _hermite_quadratic_point([-dx, 0.0, dx], mu, [], [])
    beta = np.array([_jiang_shu(p, dx, 2) for p in (p1, p2, p3)])
    dp = np.array([p.deriv()(0.0) for p in (p1, p2, p3)])
    eps = 1e-6
    wt = np.array([0.25, 0.25, 0.5]) / (beta + eps) ** 2
    ref = float(np.dot(wt / wt.sum(), dp))
    got = orc.limiter_value(mu, nu, dx, eps=eps)
    assert abs(got - ref) <= 1e-12 * max(1.0, np.max(np.abs(dp)))


@pytest.mark.parametrize("nc,direction", [(2, 0), (3, 0), (3, 1)])
def test_eigenvectors_diagonalise_flux_jacobian(orc, nc, direction):
    # L R = I, and R diag(lambda) L equals the Jacobian dF/dU of the pre-balanced flux (eq. swe-form-2d-e)
    # obtained by central differences of the oracle's own pointwise flux at fixed b.
    g = 9.812
    rng = np.random.default_rng(7 + nc + direction)
    for _ in range(5):
        h, u, v, b = rng.uniform(0.5, 2.0), rng.normal(), rng.normal(), rng.uniform(-0.5, 0.5)
        c = np.sqrt(g * h)
        L, R = orc.eigenvectors(nc, direction, u, v if nc == 3 else 0.0, c)
        np.testing.assert_allclose(L @ R, np.eye(nc), atol=1e-14)
        U0 = np.array([h + b, h * u, h * v])[:nc]

        def flux(U):
            s = np.zeros(12)
            s[0], s[1] = U[0], U[1]
            s[2] = U[2] if nc == 3 else 0.0
            s[9] = b
            out = orc.pointwise2d(g, s)
            return (out[0] if direction == 0 else out[1])[:nc]

        J = np.zeros((nc, nc))
        for k in range(nc):
            e = np.zeros(nc); e[k] = 1e-6
            J[:, k] = (flux(U0 + e) - flux(U0 - e)) / 2e-6
        un = u if direction == 0 else v
        lam = np.array([un - c, un, un + c]) if nc == 3 else np.array([un - c, un + c])
        np.testing.assert_allclose(R @ np.diag(lam) @ L, J, atol=1e-6 * max(1, np.abs(J).max()))


def test_derivative_fluxes_are_chain_rule(orc):
    # Phi1 = dF1/dx, Phi2 = dF2/dx, Psi1 = dF1/dy, Psi2 = dF2/dy (Sec. 3 after eq. swe-form-2d-h), checked by
    # central differences along smooth fields.
    g = 9.812
    def fields(x, y):
        eta = 1.3 + 0.2 * np.sin(x) * np.cos(y)
        m = 0.3 * np.cos(2 * x + y)
        w = -0.2 * np.sin(x - 3 * y)
        b = 0.4 * np.exp(-x * x - 0.5 * y * y)
        return np.array([eta, m, w, b])
    def grad(x, y, e=1e-6):
        return ((fields(x + e, y) - fields(x - e, y)) / (2 * e), (fields(x, y + e) - fields(x, y - e)) / (2 * e))
    def flux(x, y):
        eta, m, w, b = fields(x, y)
        s = np.zeros(12); s[0], s[1], s[2], s[9] = eta, m, w, b
        return orc.pointwise2d(g, s)
    for (x, y) in [(0.1, 0.2), (-0.7, 0.4), (1.1, -0.3)]:
        gx, gy = grad(x, y)
        s = np.zeros(12)
        eta, m, w, b = fields(x, y)
        s[0], s[1], s[2] = eta, m, w
        s[3], s[4], s[5] = gx[0], gx[1], gx[2]
        s[6], s[7], s[8] = gy[0], gy[1], gy[2]
        s[9], s[10], s[11] = b, gx[3], gy[3]
        out = orc.pointwise2d(g, s)
        e = 1e-6
        dFdx = (flux(x + e, y) - flux(x - e, y)) / (2 * e)
        dFdy = (flux(x, y + e) - flux(x, y - e)) / (2 * e)
        np.testing.assert_allclose(out[2], dFdx[0], atol=1e-7)  # Phi1 = d_x F1
        np.testing.assert_allclose(out[3], dFdx[1], atol=1e-7)  # Phi2 = d_x F2
        np.testing.assert_allclose(out[4], dFdy[0], atol=1e-7)  # Psi1 = d_y F1
        np.testing.assert_allclose(out[5], dFdy[1], atol=1e-7)  # Psi2 = d_y F2
