"""Gradients of a gauge-misfit loss through the hand-written discrete adjoint of the 2D scheme.

``hw_adjoint_step``, ``hw_gauge_loss`` and ``hw_adjoint_run`` are the C functions of
``include/hwswe.h`` (argument marshalling only). ``GaugeMisfit`` is a ``torch.autograd.Function``:
its forward evaluates L = sum_n sum_g (eta^n[g] - eta_obs[n-1][g])^2 of a run with given time steps
from an initial equilibrium state (9 planes) and bottom (b, b_x, b_y), and its backward calls the
adjoint (by default on a whole-run tape when it fits in device memory, else with binomial
checkpointing).
"""
from __future__ import annotations

import ctypes as C
from typing import Sequence

import numpy as np

from . import HW_LAYOUT_EQUILIBRIUM, _check, _pp, _ptr, hw_init, hw_set_state, lib

# storage modes of hw_adjoint_run besides a snapshot count (include/hwswe.h)
HW_ADJ_TAPE = -1  # keep every stage of every step: no recomputation
HW_ADJ_AUTO = -2  # the tape when it fits in device memory, else checkpointing with the snapshots that fit


def _sigs():
    L = lib()
    if getattr(L, "_adj_ready", False):
        return L
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    pp = C.POINTER(C.c_void_p)
    L.hw_adjoint_step.argtypes = [vp, d, pp, pp]
    L.hw_adjoint_step.restype = i
    L.hw_gauge_loss.argtypes = [vp, i, C.POINTER(d), C.POINTER(i), i, C.POINTER(d), C.POINTER(d), C.POINTER(d)]
    L.hw_gauge_loss.restype = i
    L.hw_adjoint_run.argtypes = [vp, i, C.POINTER(d), C.POINTER(i), i, C.POINTER(d), i, C.POINTER(d), pp, pp,
                                 C.POINTER(C.c_longlong)]
    L.hw_adjoint_run.restype = i
    L._adj_ready = True
    return L


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype).ravel())


def hw_adjoint_step(h, dt: float, lam_state: Sequence, lam_static: Sequence):
    n = h.n
    _check(_sigs().hw_adjoint_step(h.ptr, float(dt), _pp([_ptr(a, n, True) for a in lam_state]),
                                   _pp([_ptr(a, n, True) for a in lam_static])), "hw_adjoint_step")


def hw_gauge_loss(h, dts, gauge_idx, eta_obs):
    dts = _host(dts, np.float64)
    gi = _host(gauge_idx, np.int32)
    ob = _host(eta_obs, np.float64)
    loss = C.c_double()
    vals = np.zeros(len(dts) * len(gi))
    dp = C.POINTER(C.c_double)
    _check(_sigs().hw_gauge_loss(h.ptr, len(dts), dts.ctypes.data_as(dp), gi.ctypes.data_as(C.POINTER(C.c_int)),
                                 len(gi), ob.ctypes.data_as(dp), C.byref(loss), vals.ctypes.data_as(dp)),
           "hw_gauge_loss")
    return loss.value, vals.reshape(len(dts), len(gi))


def hw_adjoint_run(h, dts, gauge_idx, eta_obs, snapshots: int, grad_state: Sequence, grad_static: Sequence):
    """Loss and gradient into the given CUDA tensors; returns (loss, forward steps taken)."""
    dts = _host(dts, np.float64)
    gi = _host(gauge_idx, np.int32)
    ob = _host(eta_obs, np.float64)
    loss = C.c_double()
    nf = C.c_longlong()
    dp = C.POINTER(C.c_double)
    n = h.n
    _check(_sigs().hw_adjoint_run(h.ptr, len(dts), dts.ctypes.data_as(dp), gi.ctypes.data_as(C.POINTER(C.c_int)),
                                  len(gi), ob.ctypes.data_as(dp), int(snapshots), C.byref(loss),
                                  _pp([_ptr(a, n, True) for a in grad_state]),
                                  _pp([_ptr(a, n, True) for a in grad_static]), C.byref(nf)), "hw_adjoint_run")
    return loss.value, nf.value


def load_problem(solver, state, static):
    """Put an equilibrium state (9 planes) and a bottom (b, b_x, b_y) into a 2D solver exactly: the
    bottom through hw_init (which precomputes its source terms), the state through hw_set_state."""
    import torch
    b, bx, by = static[0], static[1], static[2]
    z = torch.zeros_like(b)
    # physical variables only matter for h > 0 here; the state is overwritten below
    hw_init(solver.h, (state[0] - b).contiguous(), state[1].contiguous(), state[2].contiguous(), b.contiguous(),
            [(state[3] - bx).contiguous(), state[4].contiguous(), state[5].contiguous(), (state[6] - by).contiguous(),
             state[7].contiguous(), state[8].contiguous(), bx.contiguous(), by.contiguous()])
    hw_set_state(solver.h, [state[q].contiguous() for q in range(9)], HW_LAYOUT_EQUILIBRIUM)
    del z


class GaugeMisfit:
    """torch.autograd.Function computing the gauge misfit of a run and its gradient by the adjoint."""

    @staticmethod
    def apply(state, static, solver, dts, gauge_idx, eta_obs, snapshots=HW_ADJ_AUTO):
        return _GaugeMisfitFn.apply(state, static, solver, dts, gauge_idx, eta_obs, snapshots)


def _make_fn():
    import torch

    class Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, state, static, solver, dts, gauge_idx, eta_obs, snapshots):
            load_problem(solver, state, static)
            loss, _ = hw_gauge_loss(solver.h, dts, gauge_idx, eta_obs)
            ctx.save_for_backward(state, static)
            ctx.args = (solver, dts, gauge_idx, eta_obs, snapshots)
            return torch.tensor(loss, dtype=torch.float64, device=state.device)

        @staticmethod
        def backward(ctx, grad_out):
            state, static = ctx.saved_tensors
            solver, dts, gauge_idx, eta_obs, snapshots = ctx.args
            load_problem(solver, state, static)
            gs = torch.empty_like(state)
            gb = torch.empty_like(static)
            hw_adjoint_run(solver.h, dts, gauge_idx, eta_obs, snapshots, [gs[q] for q in range(9)],
                           [gb[q] for q in range(3)])
            return gs * grad_out, gb * grad_out, None, None, None, None, None

    return Fn


class _Lazy:
    _fn = None

    @classmethod
    def apply(cls, *a):
        if cls._fn is None:
            cls._fn = _make_fn()
        return cls._fn.apply(*a)


_GaugeMisfitFn = _Lazy
