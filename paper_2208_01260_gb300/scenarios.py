"""Seeded synthetic inputs for the shallow water workloads.

This module produces physical initial data only: depth h, discharges hu, hv, bottom b and their
analytic first derivatives, on the node layout both sides use. It holds none of the scheme's
arithmetic (no conversion to eta = h + b, no fluxes), so the CPU oracle and the CUDA path can both
consume it without sharing any of the method.

Node layout: periodic directions put nodes at x0 + i*dx; reflective directions put them at cell
centres x0 + (i + 1/2)*dx with walls at the faces x0, x1. Arrays are float64, shape (ny, nx),
row-major with x fastest (1D: shape (nx,)).

Workloads (the paper has no dataset; these stand in for its analytic examples):
  * ``lake1d_bumps`` / ``perturbed1d``  -- 1D, N=200 on [0,2], reflective, two Gaussian bumps,
    still water eta=1 (+1e-3 on a random 0.1-wide interval). Modelled on Ex. 4.3.
  * ``accuracy1d``   -- 1D periodic smooth data of Ex. 4.1 with random phase shifts.
  * ``bumps2d``      -- 2D reflective, Gaussian bumps, eta=1 (+0.01 strip on x in [0.05, 0.15]),
    modelled on Ex. 4.8 (2048^2 on [0,2]x[0,1] for the benchmark).
  * ``hump2d``       -- 2D reflective, bumps plus a Gaussian hump of the free surface (batched and
    adjoint workloads).
  * the paper's own analytic examples: ``ex41``, ``ex42``, ``ex46``, ``ex47``, ``ex48``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

PERIODIC = 0
REFLECTIVE = 1
OUTFLOW = 2
SEED_BASE = 2208012600


@dataclass
class Scenario:
    """Physical initial data plus the grid it lives on."""
    dim: int
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    bc_x: int
    bc_y: int
    h: np.ndarray
    hu: np.ndarray
    b: np.ndarray
    deriv: List[np.ndarray]          # 2D: h_x, hu_x, hv_x, h_y, hu_y, hv_y, b_x, b_y; 1D: h_x, hu_x, b_x
    hv: Optional[np.ndarray] = None
    eps_w: float = 1e-6
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny


def axis(n: int, a: float, b: float, bc: int) -> np.ndarray:
    d = (b - a) / n
    off = 0.0 if bc == PERIODIC else 0.5
    return a + (np.arange(n, dtype=np.float64) + off) * d


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------------------------------------
# Gaussian bumps: A exp(-((x-xc)^2 + (y-yc)^2) / s^2) and their analytic derivatives
# ------------------------------------------------------------------------------------------------
def _bumps2d(X, Y, amps, xcs, ycs, sigmas):
    b = np.zeros_like(X)
    bx = np.zeros_like(X)
    by = np.zeros_like(X)
    for A, xc, yc, s in zip(amps, xcs, ycs, sigmas):
        g = A * np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / s ** 2)
        b += g
        bx += -2.0 * (X - xc) / s ** 2 * g
        by += -2.0 * (Y - yc) / s ** 2 * g
    return b, bx, by


def _bumps1d(x, amps, xcs, sigmas):
    b = np.zeros_like(x)
    bx = np.zeros_like(x)
    for A, xc, s in zip(amps, xcs, sigmas):
        g = A * np.exp(-((x - xc) ** 2) / s ** 2)
        b += g
        bx += -2.0 * (x - xc) / s ** 2 * g
    return b, bx


def _cap(b, *ders, cap=0.75):
    """Rescale the bottom so max b <= cap (keeps h >= 1 - cap under still water eta = 1)."""
    m = float(np.max(b))
    if m > cap:
        f = cap / m
        return (b * f,) + tuple(d * f for d in ders)
    return (b,) + tuple(ders)


# ------------------------------------------------------------------------------------------------
# 1D workloads
# ------------------------------------------------------------------------------------------------
def perturbed1d(n: int = 200, seed: int = SEED_BASE + 1, perturb: float = 1e-3, lake: bool = False) -> Scenario:
    """Two Gaussian bumps on [0,2] (A~U(0.1,0.4), sigma~U(0.05,0.15), xc~U(0.2,1.8)), reflective,
    still water eta=1 plus `perturb` on a random 0.1-wide interval [s, s+0.1], s~U(0,1.9)."""
    r = _rng(seed)
    amps = r.uniform(0.1, 0.4, 2)
    sig = r.uniform(0.05, 0.15, 2)
    xcs = r.uniform(0.2, 1.8, 2)
    s = r.uniform(0.0, 1.9)
    x = axis(n, 0.0, 2.0, REFLECTIVE)
    b, bx = _bumps1d(x, amps, xcs, sig)
    b, bx = _cap(b, bx)
    eta = np.ones(n)
    if not lake:
        eta = eta + np.where((x >= s) & (x <= s + 0.1), perturb, 0.0)
    h = eta - b
    # derivative of eta is 0 on both sides of the jump, so h_x = -b_x
    return Scenario(1, n, 1, 0.0, 2.0, 0.0, 1.0, REFLECTIVE, PERIODIC, h, np.zeros(n), b,
                    [-bx, np.zeros(n), bx], eps_w=1e-10 if perturb <= 1e-3 else 1e-6,
                    name="perturbed1d" if not lake else "lake1d", meta=dict(s=s))


def accuracy1d(n: int, seed: int = SEED_BASE + 2, phases: Optional[Tuple[float, float, float]] = None) -> Scenario:
    """Ex. 4.1 data with phase shifts: h = 5 + exp(cos 2pi(x-p1)), hu = sin(cos 2pi(x-p2)),
    b = sin^2(pi(x-p3)) on [0,1], periodic.

    The seeded default draws ONE phase p ~ U(0,1) and uses p1 = p2 = p3 = p, a rigid translation of
    Ex. 4.1. Independent phases steepen the data into a bore before t = 0.1 (max |eta_x| grows from
    about 10 to about 120), after which no scheme converges at fifth order."""
    if phases is None:
        r = _rng(seed)
        p = float(r.uniform(0.0, 1.0))
        phases = (p, p, p)
    p1, p2, p3 = phases
    x = axis(n, 0.0, 1.0, PERIODIC)
    tp = 2.0 * math.pi
    h = 5.0 + np.exp(np.cos(tp * (x - p1)))
    hx = -tp * np.sin(tp * (x - p1)) * np.exp(np.cos(tp * (x - p1)))
    hu = np.sin(np.cos(tp * (x - p2)))
    hux = -tp * np.sin(tp * (x - p2)) * np.cos(np.cos(tp * (x - p2)))
    b = np.sin(math.pi * (x - p3)) ** 2
    bx = math.pi * np.sin(tp * (x - p3))
    return Scenario(1, n, 1, 0.0, 1.0, 0.0, 1.0, PERIODIC, PERIODIC, h, hu, b, [hx, hux, bx],
                    name="accuracy1d", meta=dict(phases=phases))


def ex41(n: int) -> Scenario:
    """Ex. 4.1: b = sin^2(pi x), h = 5 + exp(cos 2pi x), hu = sin(cos 2pi x), periodic on [0,1]."""
    s = accuracy1d(n, phases=(0.0, 0.0, 0.0))
    s.name = "ex41"
    return s


def ex42(n: int = 200, step: bool = False) -> Scenario:
    """Ex. 4.2 lake at rest on [0,10], h + b = 10, u = 0. Smooth b = 5 exp(-0.4 (x-5)^2) (eq. b-1) or
    the step b = 4 on [4,8] (eq. b-2). The paper gives no boundary condition; reflective walls here."""
    x = axis(n, 0.0, 10.0, REFLECTIVE)
    if step:
        b = np.where((x >= 4.0) & (x <= 8.0), 4.0, 0.0)
        bx = np.zeros(n)
    else:
        b = 5.0 * np.exp(-0.4 * (x - 5.0) ** 2)
        bx = -0.8 * (x - 5.0) * b
    h = 10.0 - b
    return Scenario(1, n, 1, 0.0, 10.0, 0.0, 1.0, REFLECTIVE, PERIODIC, h, np.zeros(n), b,
                    [-bx, np.zeros(n), bx], name="ex42" + ("step" if step else "smooth"))


def ex43(n: int = 200, eps: float = 0.2, bc: int = OUTFLOW) -> Scenario:
    """Ex. 4.3 perturbed lake at rest on [0,2]: b = 0.25 (cos(10 pi (x-1.5)) + 1) on [1.4,1.6] (eq. B-5),
    h = 1 - b (+ eps on [1.1,1.2]), u = 0, to t = 0.2; eps = 0.2 or 1e-3 (the latter with epsilon 1e-10
    in the weights). The waves stay inside the domain until t = 0.2, so the boundary does not act."""
    x = axis(n, 0.0, 2.0, bc)
    inb = (x >= 1.4) & (x <= 1.6)
    b = np.where(inb, 0.25 * (np.cos(10.0 * math.pi * (x - 1.5)) + 1.0), 0.0)
    bx = np.where(inb, -2.5 * math.pi * np.sin(10.0 * math.pi * (x - 1.5)), 0.0)
    h = 1.0 - b + np.where((x >= 1.1) & (x <= 1.2), eps, 0.0)
    return Scenario(1, n, 1, 0.0, 2.0, 0.0, 1.0, bc, PERIODIC, h, np.zeros(n), b, [-bx, np.zeros(n), bx],
                    eps_w=1e-10 if eps < 0.01 else 1e-6, name="ex43_%g" % eps, meta=dict(t_end=0.2))


def ex44(n: int = 200, bc: int = OUTFLOW) -> Scenario:
    """Ex. 4.4 rarefaction and shocks over the wavy bottom b = 0.3 cos^30(pi/2 (x-1)) on [0,2] (eq. B-3),
    domain [-10,10]: h = 2 - b, u = 1 for x <= 1; h = 0.35 - b, u = 0 beyond; to t = 1."""
    x = axis(n, -10.0, 10.0, bc)
    inb = (x >= 0.0) & (x <= 2.0)
    c = np.cos(0.5 * math.pi * (x - 1.0))
    b = np.where(inb, 0.3 * c ** 30, 0.0)
    bx = np.where(inb, -0.3 * 30.0 * c ** 29 * np.sin(0.5 * math.pi * (x - 1.0)) * 0.5 * math.pi, 0.0)
    left = x <= 1.0
    h = np.where(left, 2.0, 0.35) - b
    u = np.where(left, 1.0, 0.0)
    return Scenario(1, n, 1, -10.0, 10.0, 0.0, 1.0, bc, PERIODIC, h, h * u, b, [-bx, -bx * u, bx],
                    name="ex44", meta=dict(t_end=1.0))


def ex45(n: int = 200, bc: int = OUTFLOW) -> Scenario:
    """Ex. 4.5 dam break over a rectangular bump on (0,1500): b = 8 for |x - 750| <= 1500/8, h = 20 - b
    left of 750 and 15 - b right of it, u = 0; to t = 15 and t = 60. All derivatives are zero."""
    x = axis(n, 0.0, 1500.0, bc)
    b = np.where(np.abs(x - 750.0) <= 187.5, 8.0, 0.0)
    h = np.where(x <= 750.0, 20.0, 15.0) - b
    z = np.zeros(n)
    return Scenario(1, n, 1, 0.0, 1500.0, 0.0, 1.0, bc, PERIODIC, h, z.copy(), b, [z.copy(), z.copy(), z.copy()],
                    name="ex45", meta=dict(t_end=(15.0, 60.0)))


# ------------------------------------------------------------------------------------------------
# 2D workloads
# ------------------------------------------------------------------------------------------------
def _still2d(X, Y, b, bx, by, eta, etax, etay, bc_x, bc_y, box, name, eps=1e-6, meta=None) -> Scenario:
    ny, nx = X.shape
    z = np.zeros_like(X)
    h = eta - b
    return Scenario(2, nx, ny, box[0], box[1], box[2], box[3], bc_x, bc_y, h, z.copy(), b,
                    [etax - bx, z.copy(), z.copy(), etay - by, z.copy(), z.copy(), bx, by], hv=z.copy(),
                    eps_w=eps, name=name, meta=meta or {})


def bumps2d(nx: int = 2048, ny: int = 2048, seed: int = SEED_BASE + 3, nbumps: int = 8, strip: float = 0.01,
            box=(0.0, 2.0, 0.0, 1.0), bc=REFLECTIVE, amp=(0.05, 0.5), sigma=(0.03, 0.15)) -> Scenario:
    """Gaussian bumps (A~U(amp), sigma~U(sigma), centres uniform in the box), still water eta = 1,
    plus `strip` on x in [0.05, 0.15] (Ex. 4.8's perturbation). strip = 0 gives the lake at rest."""
    r = _rng(seed)
    amps = r.uniform(amp[0], amp[1], nbumps)
    sig = r.uniform(sigma[0], sigma[1], nbumps)
    xcs = r.uniform(box[0], box[1], nbumps)
    ycs = r.uniform(box[2], box[3], nbumps)
    x = axis(nx, box[0], box[1], bc)
    y = axis(ny, box[2], box[3], bc)
    X, Y = np.meshgrid(x, y)
    b, bx, by = _bumps2d(X, Y, amps, xcs, ycs, sig)
    b, bx, by = _cap(b, bx, by)
    eta = np.ones_like(X)
    if strip:
        eta = eta + np.where((X >= 0.05) & (X <= 0.15), strip, 0.0)
    z = np.zeros_like(X)
    return _still2d(X, Y, b, bx, by, eta, z, z, bc, bc, box, "bumps2d" if strip else "lake2d")


def hump2d(nx: int, ny: int, seed: int, box=(0.0, 1.0, 0.0, 1.0), bc=REFLECTIVE, max_bumps: int = 16,
           amp_max: float = 0.6, hump_max: float = 0.05) -> Scenario:
    """K~U{1..max_bumps} Gaussian bumps (A~U(0, amp_max), sigma~U(0.03, 0.15)) and a Gaussian hump of
    the free surface eta = 1 + A_s exp(-r^2/s_s^2), A_s~U(0, hump_max), s_s~U(0.05, 0.2), with the
    hump's analytic derivatives."""
    r = _rng(seed)
    k = int(r.integers(1, max_bumps + 1))
    amps = r.uniform(0.0, amp_max, k)
    sig = r.uniform(0.03, 0.15, k)
    xcs = r.uniform(box[0], box[1], k)
    ycs = r.uniform(box[2], box[3], k)
    As = r.uniform(0.0, hump_max)
    ss = r.uniform(0.05, 0.2)
    xs = r.uniform(box[0] + 0.2 * (box[1] - box[0]), box[1] - 0.2 * (box[1] - box[0]))
    ys = r.uniform(box[2] + 0.2 * (box[3] - box[2]), box[3] - 0.2 * (box[3] - box[2]))
    x = axis(nx, box[0], box[1], bc)
    y = axis(ny, box[2], box[3], bc)
    X, Y = np.meshgrid(x, y)
    b, bx, by = _bumps2d(X, Y, amps, xcs, ycs, sig)
    b, bx, by = _cap(b, bx, by)
    g = As * np.exp(-((X - xs) ** 2 + (Y - ys) ** 2) / ss ** 2)
    eta = 1.0 + g
    etax = -2.0 * (X - xs) / ss ** 2 * g
    etay = -2.0 * (Y - ys) / ss ** 2 * g
    return _still2d(X, Y, b, bx, by, eta, etax, etay, bc, bc, box, "hump2d",
                    meta=dict(nbumps=k, hump=(As, ss, xs, ys)))


def ex46(n: int) -> Scenario:
    """Ex. 4.6: b = sin 2pi x + sin 2pi y, h = 10 + exp(sin 2pi x) cos 2pi y,
    hu = sin(cos 2pi x) sin 2pi y, hv = cos 2pi x cos(sin 2pi y), periodic on [0,1]^2."""
    x = axis(n, 0.0, 1.0, PERIODIC)
    X, Y = np.meshgrid(x, x)
    tp = 2.0 * math.pi
    sx, cx, sy, cy = np.sin(tp * X), np.cos(tp * X), np.sin(tp * Y), np.cos(tp * Y)
    b = sx + sy
    bx, by = tp * cx, tp * cy
    h = 10.0 + np.exp(sx) * cy
    hx = tp * cx * np.exp(sx) * cy
    hy = -tp * np.exp(sx) * sy
    hu = np.sin(cx) * sy
    hux = -tp * sx * np.cos(cx) * sy
    huy = tp * np.sin(cx) * cy
    hv = cx * np.cos(sy)
    hvx = -tp * sx * np.cos(sy)
    hvy = -tp * cx * np.sin(sy) * cy
    return Scenario(2, n, n, 0.0, 1.0, 0.0, 1.0, PERIODIC, PERIODIC, h, hu, b,
                    [hx, hux, hvx, hy, huy, hvy, bx, by], hv=hv, name="ex46")


def ex47(n: int = 200) -> Scenario:
    """Ex. 4.7: b = 0.8 exp(-50((x-0.5)^2 + (y-0.5)^2)), h = 1 - b, u = v = 0, periodic on [0,1]^2."""
    x = axis(n, 0.0, 1.0, PERIODIC)
    X, Y = np.meshgrid(x, x)
    b = 0.8 * np.exp(-50.0 * ((X - 0.5) ** 2 + (Y - 0.5) ** 2))
    bx = -100.0 * (X - 0.5) * b
    by = -100.0 * (Y - 0.5) * b
    z = np.zeros_like(X)
    return _still2d(X, Y, b, bx, by, np.ones_like(X), z, z, PERIODIC, PERIODIC, (0.0, 1.0, 0.0, 1.0), "ex47")


def ex48(nx: int = 200, ny: int = 100, bc=REFLECTIVE) -> Scenario:
    """Ex. 4.8: b = 0.8 exp(-5(x-0.9)^2 - 50(y-0.5)^2) on [0,2]x[0,1], h = 1 - b (+0.01 on
    x in [0.05, 0.15]), u = v = 0. The paper states no boundary condition; reflective walls here."""
    x = axis(nx, 0.0, 2.0, bc)
    y = axis(ny, 0.0, 1.0, bc)
    X, Y = np.meshgrid(x, y)
    b = 0.8 * np.exp(-5.0 * (X - 0.9) ** 2 - 50.0 * (Y - 0.5) ** 2)
    bx = -10.0 * (X - 0.9) * b
    by = -100.0 * (Y - 0.5) * b
    eta = 1.0 + np.where((X >= 0.05) & (X <= 0.15), 0.01, 0.0)
    z = np.zeros_like(X)
    return _still2d(X, Y, b, bx, by, eta, z, z, bc, bc, (0.0, 2.0, 0.0, 1.0), "ex48")


def ex49(n: int = 200, bc: int = OUTFLOW) -> Scenario:
    """Ex. 4.9 circular dam break on [0,2]^2: b = (cos(2 pi (x-0.5)) + 1)(cos(2 pi y) + 1) / 8 inside the
    circle of radius 0.5 about (1.5, 1) (zero outside), h = 1.1 - b inside the circle of radius 0.1
    about (1.25, 1) and 0.6 - b elsewhere, u = v = 0; to t = 0.15 (the waves stay inside the domain)."""
    x = axis(n, 0.0, 2.0, bc)
    X, Y = np.meshgrid(x, x)
    inb = np.hypot(X - 1.5, Y - 1.0) <= 0.5
    cx, cy = np.cos(2.0 * math.pi * (X - 0.5)) + 1.0, np.cos(2.0 * math.pi * Y) + 1.0
    b = np.where(inb, cx * cy / 8.0, 0.0)
    bx = np.where(inb, -2.0 * math.pi * np.sin(2.0 * math.pi * (X - 0.5)) * cy / 8.0, 0.0)
    by = np.where(inb, -2.0 * math.pi * np.sin(2.0 * math.pi * Y) * cx / 8.0, 0.0)
    eta = np.where(np.hypot(X - 1.25, Y - 1.0) <= 0.1, 1.1, 0.6)
    z = np.zeros_like(X)
    return _still2d(X, Y, b, bx, by, eta, z, z, bc, bc, (0.0, 2.0, 0.0, 2.0), "ex49", meta=dict(t_end=0.15))


def adjoint_case(n: int = 512, seed: int = SEED_BASE + 5, hump_seed: int = 0) -> Scenario:
    """Adjoint workload: the benchmark's bottom (8 Gaussian bumps on [0,2]x[0,1], reflective) at n x n
    without the strip, plus a Gaussian hump of the surface (amplitude U(0.02, 0.05), width U(0.05, 0.1),
    centre in the interior) drawn from ``hump_seed`` (0 for the model, others for observation runs)."""
    sc = bumps2d(n, n, seed=seed, strip=0.0)
    r = _rng(seed * 7 + 1000 + hump_seed)
    A = r.uniform(0.02, 0.05)
    s_ = r.uniform(0.05, 0.1)
    xc = r.uniform(0.4, 1.6)
    yc = r.uniform(0.3, 0.7)
    x = axis(sc.nx, sc.x0, sc.x1, sc.bc_x)
    y = axis(sc.ny, sc.y0, sc.y1, sc.bc_y)
    X, Y = np.meshgrid(x, y)
    g = A * np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / s_ ** 2)
    sc.h = sc.h + g
    sc.deriv[0] = sc.deriv[0] - 2.0 * (X - xc) / s_ ** 2 * g
    sc.deriv[3] = sc.deriv[3] - 2.0 * (Y - yc) / s_ ** 2 * g
    sc.name = "adjoint%d" % hump_seed
    sc.meta = dict(hump=(A, s_, xc, yc))
    return sc


def gauges(nx: int, ny: int, count: int = 32, seed: int = SEED_BASE + 6):
    """Seeded gauge nodes (linear indices j*nx + i), distinct."""
    r = _rng(seed)
    return np.sort(r.choice(nx * ny, count, replace=False)).astype(np.int32)


def batch_sizes(n: int = 512, seed: int = SEED_BASE + 4, lo: int = 64, hi: int = 1024):
    """Grid sizes nx, ny independently log-uniform integers on [lo, hi]."""
    r = _rng(seed)
    nx = np.exp(r.uniform(math.log(lo), math.log(hi), n)).round().astype(int)
    ny = np.exp(r.uniform(math.log(lo), math.log(hi), n)).round().astype(int)
    return np.clip(nx, lo, hi), np.clip(ny, lo, hi)


def batch_scenario(i: int, nx: int, ny: int, seed: int = SEED_BASE + 4) -> Scenario:
    """Instance i of the batched workload: hump2d on [0,1]^2 with its own seed."""
    s = hump2d(nx, ny, seed * 1000 + i)
    s.name = "batch%d" % i
    return s


def random_sample(nx: int, ny: int, count: int, seed: int):
    """Seeded node sample (i, j) that always includes the four corners and the wall-adjacent nodes."""
    r = _rng(seed)
    pi = list(r.integers(0, nx, count))
    pj = list(r.integers(0, ny, count))
    for (a, b) in [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1), (1, 1), (nx - 2, ny - 2),
                   (0, ny // 2), (nx // 2, 0), (nx - 1, ny // 2), (nx // 2, ny - 1)]:
        pi.append(a)
        pj.append(b)
    return np.array(pi, dtype=np.int32), np.array(pj, dtype=np.int32)
