"""CPU oracle for the well-balanced fifth-order FD HWENO scheme (Zhao & Zhang, arXiv:2208.01260).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. The CUDA library never imports or links it, and it imports
nothing from the CUDA package.

The arithmetic lives in ``hwswe_oracle.cpp`` (plain FP64 C++, ghost-padded arrays, the paper's
formulas in the paper's order; see its header for the sections each part follows and the readings
taken where the paper is silent or garbled). This module compiles it with g++ and wraps its C
functions with ctypes and numpy.

Parity pins (all in ``tests/test_oracle_*.py``): polynomial exactness of the Hermite candidates,
of the quintic Q and of its derivative; the smoothness indicators against their integral
definition; the limiter's linear combination; L R = I and R diag(lambda) L = dF/dU; Phi = dF/dx;
lake at rest to round-off; fifth-order truncation and convergence; mirror and transpose symmetry;
2D reducing to 1D; mass conservation. The nonlinear weights at discontinuities have no closed form:
there the oracle is pinned only through these invariants.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hwswe_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC = 0
BC_REFLECTIVE = 1
BC_OUTFLOW = 2  # transmissive: ghosts copy the boundary node


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("bc_x", C.c_int), ("bc_y", C.c_int)]


class Params(C.Structure):
    _fields_ = [("g", C.c_double), ("cfl", C.c_double), ("eps_w", C.c_double), ("eps_lim", C.c_double),
                ("char_decomp", C.c_int), ("limiter", C.c_int), ("linear_weights", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (g++, -O2, no FP contraction, OpenMP)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        pp = C.POINTER(dp)
        gp, prp = C.POINTER(Grid), C.POINTER(Params)
        for name, args, res in [
            ("orc_candidates", [dp, dp, C.c_double, dp], None),
            ("orc_smoothness", [dp, dp, C.c_double, dp], None),
            ("orc_hweno_value", [dp, dp, C.c_double, C.c_double, C.c_int, dp], C.c_double),
            ("orc_qprime", [dp, dp, C.c_double], C.c_double),
            ("orc_limiter_value", [dp, dp, C.c_double, C.c_double, C.c_int], C.c_double),
            ("orc_eigenvectors", [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, dp, dp], None),
            ("orc_pointwise2d", [C.c_double, dp, dp], None),
            ("orc_alpha2d", [gp, prp, pp, pp, dp], C.c_int),
            ("orc_rhs2d", [gp, prp, pp, pp, pp, dp], C.c_int),
            ("orc_rhs2d_f32", [gp, prp, pp, pp, pp, dp], C.c_int),
            ("orc_limiter2d", [gp, prp, pp, pp, pp], C.c_int),
            ("orc_stage2d", [gp, prp, C.c_int, C.c_double, pp, pp, pp, pp, dp], C.c_int),
            ("orc_stage2d_f32", [gp, prp, C.c_int, C.c_double, pp, pp, pp, pp, dp], C.c_int),
            ("orc_stage2d_points", [gp, prp, C.c_int, C.c_double, pp, pp, dp, C.c_int, ip, ip, dp, dp, dp],
             C.c_int),
            ("orc_rk3_step2d", [gp, prp, C.c_double, pp, pp], C.c_int),
            ("orc_cfl_dt2d", [gp, prp, pp, pp], C.c_double),
            ("orc_count_stage2d", [gp, prp, pp, pp, dp], C.c_int),
            ("orc_alpha1d", [gp, prp, pp, pp, dp], C.c_int),
            ("orc_rhs1d", [gp, prp, pp, pp, pp, dp], C.c_int),
            ("orc_limiter1d", [gp, prp, pp, pp, pp], C.c_int),
            ("orc_stage1d", [gp, prp, C.c_int, C.c_double, pp, pp, pp, pp, dp], C.c_int),
            ("orc_rk3_step1d", [gp, prp, C.c_double, pp, pp], C.c_int),
            ("orc_cfl_dt1d", [gp, prp, pp, pp], C.c_double),
            ("orc_gauge_loss_dual2d", [gp, prp, pp, pp, pp, pp, C.c_int, dp, ip, C.c_int, dp, dp], C.c_int),
            ("orc_lake_run", [gp, prp, pp, pp, C.c_double, C.c_int, dp, ip], C.c_int),
        ]:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


# ------------------------------------------------------------------------------------------------
# helpers
# ------------------------------------------------------------------------------------------------
def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _arr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptrs(planes):
    arrs = [np.ascontiguousarray(p, dtype=np.float64) for p in planes]
    P = (C.POINTER(C.c_double) * len(arrs))(*[_d(a) for a in arrs])
    return P, arrs


def make_grid(nx, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x=BC_PERIODIC, bc_y=BC_PERIODIC, dim=None):
    if dim is None:
        dim = 1 if ny == 1 else 2
    return Grid(dim, nx, ny, x0, x1, y0, y1, bc_x, bc_y)


def make_params(g=9.812, cfl=0.6, eps_w=1e-6, eps_lim=None, char_decomp=1, limiter=1, linear_weights=0):
    return Params(g, cfl, eps_w, eps_w if eps_lim is None else eps_lim, char_decomp, limiter, linear_weights)


def node_coords(grid):
    """Node positions: periodic x_i = x0 + i dx; reflective cell-centred x_i = x0 + (i+1/2) dx."""
    dx = (grid.x1 - grid.x0) / grid.nx
    x = grid.x0 + (np.arange(grid.nx) + (0.0 if grid.bc_x == BC_PERIODIC else 0.5)) * dx
    if grid.dim == 1:
        return x
    dy = (grid.y1 - grid.y0) / grid.ny
    y = grid.y0 + (np.arange(grid.ny) + (0.0 if grid.bc_y == BC_PERIODIC else 0.5)) * dy
    return x, y


# ------------------------------------------------------------------------------------------------
# physical <-> equilibrium variables (Sec. 2 and 3: eta = h + b, derivatives of eta = h_x + b_x)
# ------------------------------------------------------------------------------------------------
def to_state2d(h, hu, hv, b, deriv):
    """deriv = (h_x, hu_x, hv_x, h_y, hu_y, hv_y, b_x, b_y) -> state planes (9) and static (3)."""
    hx, hux, hvx, hy, huy, hvy, bx, by = deriv
    st = [h + b, hu, hv, hx + bx, hux, hvx, hy + by, huy, hvy]
    return [np.array(p, dtype=np.float64) for p in st], [np.array(p, dtype=np.float64) for p in (b, bx, by)]


def to_state1d(h, hu, b, deriv):
    """deriv = (h_x, hu_x, b_x) -> state planes (4) and static (2)."""
    hx, hux, bx = deriv
    return ([np.array(p, dtype=np.float64) for p in (h + b, hu, hx + bx, hux)],
            [np.array(p, dtype=np.float64) for p in (b, bx)])


# ------------------------------------------------------------------------------------------------
# scalar pieces
# ------------------------------------------------------------------------------------------------
def candidates(f, phi, dx):
    f, phi = _arr(f), _arr(phi)
    q = np.zeros(3)
    lib().orc_candidates(_d(f), _d(phi), dx, _d(q))
    return q


def smoothness(f, phi, dx):
    f, phi = _arr(f), _arr(phi)
    b = np.zeros(3)
    lib().orc_smoothness(_d(f), _d(phi), dx, _d(b))
    return b


def hweno_value(f, phi, dx, eps=1e-6, linear=False):
    f, phi = _arr(f), _arr(phi)
    w = np.zeros(3)
    v = lib().orc_hweno_value(_d(f), _d(phi), dx, eps, int(linear), _d(w))
    return v, w


def qprime(f, phi, dx):
    f, phi = _arr(f), _arr(phi)
    return lib().orc_qprime(_d(f), _d(phi), dx)


def limiter_value(mu, nu, dx, eps=1e-6, linear=False):
    mu, nu = _arr(mu), _arr(nu)
    return lib().orc_limiter_value(_d(mu), _d(nu), dx, eps, int(linear))


def eigenvectors(nc, direction, u, v, c):
    L = np.zeros(nc * nc)
    R = np.zeros(nc * nc)
    lib().orc_eigenvectors(nc, direction, u, v, c, _d(L), _d(R))
    return L.reshape(nc, nc), R.reshape(nc, nc)


def pointwise2d(g, s12):
    s12 = _arr(s12)
    out = np.zeros(18)
    lib().orc_pointwise2d(g, _d(s12), _d(out))
    return out.reshape(6, 3)  # F1, F2, Phi1, Phi2, Psi1, Psi2


# ------------------------------------------------------------------------------------------------
# 2D scheme
# ------------------------------------------------------------------------------------------------
def _check(rc, name):
    if rc != 0:
        raise ValueError("%s rejected its arguments" % name)


def alpha2d(grid, params, st, stat):
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    out = np.zeros(2)
    _check(lib().orc_alpha2d(C.byref(grid), C.byref(params), S, T, _d(out)), "orc_alpha2d")
    return out


def rhs2d(grid, params, st, stat, single=False):
    """Right-hand side (9 planes) and alpha; single=True computes every operation in float."""
    shape = (grid.ny, grid.nx)
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    outs = [np.zeros(shape) for _ in range(9)]
    O, o = _ptrs(outs)
    al = np.zeros(2)
    fn = lib().orc_rhs2d_f32 if single else lib().orc_rhs2d
    _check(fn(C.byref(grid), C.byref(params), S, T, O, _d(al)), "orc_rhs2d")
    return o, al


def limiter2d(grid, params, st, stat):
    shape = (grid.ny, grid.nx)
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    outs = [np.zeros(shape) for _ in range(6)]
    O, o = _ptrs(outs)
    _check(lib().orc_limiter2d(C.byref(grid), C.byref(params), S, T, O), "orc_limiter2d")
    return o


def stage2d(grid, params, k, dt, st, stat, base=None, single=False):
    """One SSP-RK3 stage. Returns (out planes, base planes, alpha). base is produced at k == 1.
    single=True computes every operation in float (inputs rounded to float, outputs widened)."""
    shape = (grid.ny, grid.nx)
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    if base is None:
        base = [np.zeros(shape) for _ in range(9)]
    B, bb = _ptrs([np.array(x, dtype=np.float64, copy=True) for x in base])
    O, o = _ptrs([np.zeros(shape) for _ in range(9)])
    al = np.zeros(2)
    fn = lib().orc_stage2d_f32 if single else lib().orc_stage2d
    _check(fn(C.byref(grid), C.byref(params), k, dt, S, T, B, O, _d(al)), "orc_stage2d")
    return o, bb, al


def stage2d_points(grid, params, k, dt, st, stat, alpha, pi, pj, base_pts=None):
    """Stage output at selected nodes. Returns (out[npts, 9], mod[npts, 6])."""
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    n = len(pi)
    al = _arr(alpha)
    bp = _arr(base_pts if base_pts is not None else np.zeros((n, 9)))
    out = np.zeros((n, 9))
    mod = np.zeros((n, 6))
    ipt = C.POINTER(C.c_int)
    _check(lib().orc_stage2d_points(C.byref(grid), C.byref(params), k, dt, S, T, _d(al), n,
                                    pi.ctypes.data_as(ipt), pj.ctypes.data_as(ipt), _d(bp), _d(out), _d(mod)),
           "orc_stage2d_points")
    return out, mod


def rk3_step2d(grid, params, dt, st, stat):
    cur = [np.array(p, dtype=np.float64, copy=True) for p in st]
    S, c = _ptrs(cur)
    T, b = _ptrs(stat)
    _check(lib().orc_rk3_step2d(C.byref(grid), C.byref(params), dt, S, T), "orc_rk3_step2d")
    return c


def cfl_dt2d(grid, params, st, stat):
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    return lib().orc_cfl_dt2d(C.byref(grid), C.byref(params), S, T)


def count_stage2d(grid, params, st, stat):
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    out = np.zeros(5)
    _check(lib().orc_count_stage2d(C.byref(grid), C.byref(params), S, T, _d(out)), "orc_count_stage2d")
    return dict(zip(["add", "mul", "div", "sqrt", "cmp"], out.tolist()))


def run2d(grid, params, st, stat, t_end, max_steps=10**9, dt_fn=None):
    """Advance with the CFL step; the step that reaches t_end (within a relative 1e-12) is shortened to
    end exactly on it (the paper does not say how the last step ends). Returns (state, t, steps)."""
    cur = [np.array(p, dtype=np.float64, copy=True) for p in st]
    t, n = 0.0, 0
    while t < t_end and n < max_steps:
        dt = cfl_dt2d(grid, params, cur, stat) if dt_fn is None else dt_fn(cur)
        last = dt >= (t_end - t) - 1e-12 * t_end
        if last:
            dt = t_end - t
        cur = rk3_step2d(grid, params, dt, cur, stat)
        t = t_end if last else t + dt
        n += 1
    return cur, t, n


def gauge_loss_dual2d(grid, params, st, stat, dst, dstat, dts, gauge_idx, obs):
    """Gauge misfit sum_n sum_g (eta^n[g] - obs[n-1][g])^2 of the run with time steps dts, and its
    derivative along the direction (dst: 9 state planes, dstat: b, b_x, b_y) by dual numbers."""
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    DS, c = _ptrs(dst)
    DT, d = _ptrs(dstat)
    dts = _arr(dts)
    gi = np.ascontiguousarray(gauge_idx, dtype=np.int32)
    ob = _arr(obs)
    out = np.zeros(2)
    _check(lib().orc_gauge_loss_dual2d(C.byref(grid), C.byref(params), S, T, DS, DT, len(dts), _d(dts),
                                       gi.ctypes.data_as(C.POINTER(C.c_int)), len(gi), _d(ob), _d(out)),
           "orc_gauge_loss_dual2d")
    return out[0], out[1]


PRECISION = {"single": 0, "double": 1, "double-double": 2}


def lake_run(grid, params, st, stat, t_end, precision="double"):
    """Run to t_end at the CFL step in single, double or double-double precision and return the L1 and
    Linf deviations from the initial state ([h_L1, h_Linf, hu_L1, hu_Linf(, hv_L1, hv_Linf)]) and the
    step count (Sec. 4, Tables 1-3)."""
    nq = 3 if grid.dim == 2 else 2
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    out = np.zeros(2 * nq)
    steps = C.c_int(0)
    _check(lib().orc_lake_run(C.byref(grid), C.byref(params), S, T, float(t_end), PRECISION[precision], _d(out),
                              C.byref(steps)), "orc_lake_run")
    return out, steps.value


# ------------------------------------------------------------------------------------------------
# 1D scheme
# ------------------------------------------------------------------------------------------------
def alpha1d(grid, params, st, stat):
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    out = np.zeros(1)
    _check(lib().orc_alpha1d(C.byref(grid), C.byref(params), S, T, _d(out)), "orc_alpha1d")
    return float(out[0])


def rhs1d(grid, params, st, stat):
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    O, o = _ptrs([np.zeros(grid.nx) for _ in range(4)])
    al = np.zeros(1)
    _check(lib().orc_rhs1d(C.byref(grid), C.byref(params), S, T, O, _d(al)), "orc_rhs1d")
    return o, float(al[0])


def limiter1d(grid, params, st, stat):
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    O, o = _ptrs([np.zeros(grid.nx) for _ in range(2)])
    _check(lib().orc_limiter1d(C.byref(grid), C.byref(params), S, T, O), "orc_limiter1d")
    return o


def stage1d(grid, params, k, dt, st, stat, base=None):
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    if base is None:
        base = [np.zeros(grid.nx) for _ in range(4)]
    B, bb = _ptrs([np.array(x, dtype=np.float64, copy=True) for x in base])
    O, o = _ptrs([np.zeros(grid.nx) for _ in range(4)])
    al = np.zeros(1)
    _check(lib().orc_stage1d(C.byref(grid), C.byref(params), k, dt, S, T, B, O, _d(al)), "orc_stage1d")
    return o, bb, float(al[0])


def rk3_step1d(grid, params, dt, st, stat):
    cur = [np.array(p, dtype=np.float64, copy=True) for p in st]
    S, c = _ptrs(cur)
    T, b = _ptrs(stat)
    _check(lib().orc_rk3_step1d(C.byref(grid), C.byref(params), dt, S, T), "orc_rk3_step1d")
    return c


def cfl_dt1d(grid, params, st, stat):
    S, a = _ptrs(st)
    T, b = _ptrs(stat)
    return lib().orc_cfl_dt1d(C.byref(grid), C.byref(params), S, T)


def run1d(grid, params, st, stat, t_end, max_steps=10**9, dt_fn=None):
    cur = [np.array(p, dtype=np.float64, copy=True) for p in st]
    t, n = 0.0, 0
    while t < t_end and n < max_steps:
        dt = cfl_dt1d(grid, params, cur, stat) if dt_fn is None else dt_fn(cur)
        last = dt >= (t_end - t) - 1e-12 * t_end
        if last:
            dt = t_end - t
        cur = rk3_step1d(grid, params, dt, cur, stat)
        t = t_end if last else t + dt
        n += 1
    return cur, t, n
