"""Shared helpers of the parity tests (GPU path against the CPU oracle).

Tolerances (derived in the design notes from the arithmetic):
  * stage outputs, normwise per variable group G in {U, V, Q}:
        max|gpu - oracle| / max(max|oracle_G|, s_G) <= 1e-12,
    s_U = max|eta|, s_V = s_Q = max|eta| * max(|b_x|, |b_y|, 1) (pointwise relative error is meaningless
    where m ~ 0 and where the nonlinear weights are ill-conditioned);
  * right-hand sides: the same norm with the flux scales of one difference quotient,
        s_RU = g max|eta|^2 / min(dx, dy),  s_RV = s_RQ = g max|eta| max(|V|, |Q|, |b_x|, |b_y|, 1) / min(dx, dy);
  * after many steps: relative L1 per group sum|gpu - oracle| / sum|oracle| <= 1e-9 (1e-8 for
    discontinuous data).
"""
import dataclasses
import numpy as np
from paper_2208_01260_gb300 import scenarios as S

G = 9.812


def groups(nstate):
    return [(0, 3), (3, 6), (6, 9)] if nstate == 9 else [(0, 2), (2, 4)]


def stage_scales(state, stat):
    n = len(state)
    eta = np.abs(state[0]).max()
    bmax = max(np.abs(stat[1]).max(), np.abs(stat[2]).max() if len(stat) > 2 else 0.0, 1.0)
    return [eta, eta * bmax, eta * bmax][: len(groups(n))]


def rhs_scales(state, stat, dmin):
    n = len(state)
    eta = np.abs(state[0]).max()
    dmax = max([np.abs(p).max() for p in state[(3 if n == 9 else 2):]] + [np.abs(p).max() for p in stat[1:]] + [1.0])
    sU = G * eta * eta / dmin
    sV = G * eta * dmax / dmin
    return [sU, sV, sV][: len(groups(n))]


def normwise(gpu, orc, scales):
    errs = []
    for (a, b), s in zip(groups(len(orc)), scales):
        num = max(np.abs(np.asarray(gpu[q]) - np.asarray(orc[q])).max() for q in range(a, b))
        den = max(max(np.abs(np.asarray(orc[q])).max() for q in range(a, b)), s)
        errs.append(num / den)
    return errs


def rel_l1(gpu, orc):
    errs = []
    for (a, b) in groups(len(orc)):
        num = sum(np.abs(np.asarray(gpu[q]) - np.asarray(orc[q])).sum() for q in range(a, b))
        den = sum(np.abs(np.asarray(orc[q])).sum() for q in range(a, b))
        errs.append(num / max(den, 1e-300))
    return errs


def grid_kwargs(sc):
    return dict(nx=sc.nx, ny=sc.ny, x0=sc.x0, x1=sc.x1, y0=sc.y0, y1=sc.y1, bc_x=sc.bc_x, bc_y=sc.bc_y)


def oracle_grid(orc, sc):
    if sc.dim == 1:
        return orc.make_grid(sc.nx, 1, sc.x0, sc.x1, bc_x=sc.bc_x)
    return orc.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y)


def oracle_state(orc, sc):
    if sc.dim == 1:
        return orc.to_state1d(sc.h, sc.hu, sc.b, sc.deriv)
    return orc.to_state2d(sc.h, sc.hu, sc.hv, sc.b, sc.deriv)


def tiny_derivatives(sc, scale=1e-160):
    """The left half of the domain with every derivative plane scaled to ~1e-160: squares and products
    of the projected derivative data there underflow, so the kernels' integer-pipe products leave their
    fast path and those interfaces and nodes are recomputed on the FP64 pipe."""
    x = S.axis(sc.nx, sc.x0, sc.x1, sc.bc_x)
    f = np.where(x < 0.5 * (sc.x0 + sc.x1), scale, 1.0)[None, :]
    return dataclasses.replace(sc, deriv=[d * f for d in sc.deriv], name=sc.name + "_tiny_derivs")
