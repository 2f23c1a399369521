"""GB300 (sm_103a) well-balanced fifth-order FD HWENO solver for the shallow water equations.

Python binding of the C ABI in ``include/hwswe.h``: the functions below have the C names and do
argument marshalling only (numpy arrays go as host pointers, torch CUDA tensors as device
pointers, the stream is torch's current stream). Every step of the scheme runs in the CUDA
library ``libhwswe.so`` built from ``csrc/``; there is no CPU fallback: if the library is missing
the first call raises.

Scheme: Zhao & Zhang, arXiv:2208.01260 (Sec. 2 one-dimensional, Sec. 3 two-dimensional).

Typical use::

    import paper_2208_01260_gb300 as hw
    from paper_2208_01260_gb300 import scenarios as S
    s = hw.Solver.from_scenario(S.bumps2d(512, 256), hw.make_params())   # FP64; precision=hw.HW_FP32
    t, n = s.advance(10 ** 6, t_end=0.1)                                # CFL steps, CUDA graph
    eta, m, w = s.state()[:3]                                           # equilibrium layout

``BatchedSolver`` advances many grids together; ``adjoint`` holds the gradient of a gauge misfit
(``GaugeMisfit`` is a torch.autograd.Function); ``autotune`` picks the batched tile shapes.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

__all__ = [
    "HW_OK", "HW_BC_PERIODIC", "HW_BC_REFLECTIVE", "HW_BC_OUTFLOW", "HW_FP64", "HW_FP32", "HW_HOST", "HW_DEVICE",
    "HW_LAYOUT_PHYSICAL",
    "HW_LAYOUT_EQUILIBRIUM", "HwError", "hw_grid", "hw_params", "lib", "make_grid", "make_params",
    "hw_create", "hw_destroy", "hw_init", "hw_rhs", "hw_alpha", "hw_cfl_dt", "hw_rk3_step", "hw_rk3_stage",
    "hw_advance", "hw_get_state", "hw_set_state", "hw_get_base", "hw_sync", "hw_version", "Solver",
    "hw_set_profiling", "hw_get_profile", "hw_get_time", "hw_set_time", "hw_rhs1d_noalloc", "hw_selftest_fp64_int", "hw_measure_fp64_peak", "BatchedSolver", "hw_batch_create",
    "hw_batch_destroy", "hw_batch_init", "hw_batch_run", "hw_batch_get_state", "hw_batch_get_time",
    "hw_batch_set_tiles", "hw_batch_get_tiles", "hw_batch_time_tiles", "hw_batch_set_persistent",
    "hw_batch_get_persistent", "hw_batch_test_barrier_timeout", "hw_batch_get_phase_times",
    "hw_part_info", "hw_dd_partition", "hw_part_create", "hw_part_init", "hw_part_finish_init", "hw_halo_strip_size",
    "hw_halo_pack", "hw_halo_unpack", "hw_part_alpha_keys", "hw_part_stage", "hw_dd_create", "hw_dd_init",
    "hw_dd_advance", "hw_dd_get_state", "hw_dd_destroy", "hw_dd_max_keys", "hw_dd_adjoint_run", "DecomposedSolver", "PartAdjoint",
]

HW_OK = 0
HW_ERR = {-1: "HW_ERR_ARG", -2: "HW_ERR_DEPTH", -3: "HW_ERR_NONFINITE", -4: "HW_ERR_CUDA", -5: "HW_ERR_TIMEOUT",
          -6: "HW_ERR_STATE", -7: "HW_ERR_NOMEM"}
HW_BC_PERIODIC = 0
HW_BC_REFLECTIVE = 1
HW_BC_OUTFLOW = 2
HW_HOST = 0
HW_DEVICE = 1
HW_LAYOUT_PHYSICAL = 0
HW_LAYOUT_EQUILIBRIUM = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhwswe.so")
_lib = None


class HwError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__("%s failed: %s (%s)" % (where, HW_ERR.get(code, str(code)), msg))
        self.code = code


class hw_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("bc_x", C.c_int), ("bc_y", C.c_int)]


class hw_params(C.Structure):
    _fields_ = [("g", C.c_double), ("cfl", C.c_double), ("eps_w", C.c_double), ("eps_lim", C.c_double),
                ("char_decomp", C.c_int), ("limiter", C.c_int), ("linear_weights", C.c_int),
                ("precision", C.c_int)]


def lib():
    """Load libhwswe.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhwswe.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, dp, i = C.c_void_p, C.POINTER(C.c_double), C.c_int
        pp = C.POINTER(C.c_void_p)
        sigs = {
            "hw_create": ([C.POINTER(hw_grid), C.POINTER(hw_params), vp, C.POINTER(vp)], i),
            "hw_destroy": ([vp], i),
            "hw_init": ([vp, vp, vp, vp, vp, pp, i], i),
            "hw_rhs": ([vp, pp, i], i),
            "hw_alpha": ([vp, dp], i),
            "hw_cfl_dt": ([vp, dp], i),
            "hw_rk3_step": ([vp, C.c_double], i),
            "hw_rk3_stage": ([vp, i, C.c_double], i),
            "hw_advance": ([vp, i, C.c_double, i, dp, C.POINTER(C.c_int)], i),
            "hw_get_state": ([vp, pp, i, i], i),
            "hw_set_state": ([vp, pp, i, i], i),
            "hw_get_base": ([vp, pp, i], i),
            "hw_sync": ([vp], i),
            "hw_set_profiling": ([vp, i], i),
            "hw_get_profile": ([vp, dp, C.POINTER(C.c_int)], i),
            "hw_get_time": ([vp, dp, C.POINTER(C.c_longlong)], i),
            "hw_set_time": ([vp, C.c_double, C.c_longlong], i),
            "hw_selftest_fp64_int": ([i, C.c_longlong, C.c_ulonglong, C.POINTER(C.c_longlong)], i),
            "hw_measure_fp64_peak": ([i, dp], i),
            "hw_last_error": ([], C.c_char_p),
            "hw_version": ([], C.c_char_p),
        }
        for name, (args, res) in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != HW_OK:
        raise HwError(rc, where, lib().hw_last_error().decode())


def make_grid(nx, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x=HW_BC_PERIODIC, bc_y=HW_BC_PERIODIC, dim=None):
    if dim is None:
        dim = 1 if ny == 1 else 2
    return hw_grid(dim, nx, ny, x0, x1, y0, y1, bc_x, bc_y)


HW_FP64 = 0
HW_FP32 = 1


def make_params(g=9.812, cfl=0.6, eps_w=1e-6, eps_lim=None, char_decomp=1, limiter=1, linear_weights=0,
                precision=HW_FP64):
    return hw_params(g, cfl, eps_w, eps_w if eps_lim is None else eps_lim, char_decomp, limiter, linear_weights,
                     precision)


# ------------------------------------------------------------------------------------------------
# marshalling helpers
# ------------------------------------------------------------------------------------------------
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _kind(arrays) -> int:
    kinds = set()
    for a in arrays:
        if a is None:
            continue
        if _is_torch(a):
            if not a.is_cuda:
                raise ValueError("torch tensors must live on the GPU")
            kinds.add(HW_DEVICE)
        else:
            kinds.add(HW_HOST)
    if len(kinds) != 1:
        raise ValueError("pass either all numpy arrays (host) or all CUDA tensors (device)")
    return kinds.pop()


def _ptr(a, n: int, writable: bool = False):
    if a is None:
        return None
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
            raise ValueError("device planes must be contiguous float64 tensors of %d elements" % n)
        return C.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != n:
        raise ValueError("host planes must be C-contiguous float64 numpy arrays of %d elements" % n)
    if writable and not a.flags["WRITEABLE"]:
        raise ValueError("output array is read-only")
    return C.c_void_p(a.ctypes.data)


def _pp(ptrs):
    return (C.c_void_p * len(ptrs))(*[p.value if p is not None else None for p in ptrs])


def _stream_handle(stream) -> Optional[int]:
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


# ------------------------------------------------------------------------------------------------
# C names
# ------------------------------------------------------------------------------------------------
class _Handle:
    def __init__(self, ptr, grid, params, n, nstate):
        self.ptr, self.grid, self.params, self.n, self.nstate = ptr, grid, params, n, nstate


def hw_create(grid: hw_grid, params: hw_params, stream=None) -> _Handle:
    out = C.c_void_p()
    _check(lib().hw_create(C.byref(grid), C.byref(params), _stream_handle(stream), C.byref(out)), "hw_create")
    n = grid.nx * (grid.ny if grid.dim == 2 else 1)
    return _Handle(out, grid, params, n, 9 if grid.dim == 2 else 4)


def hw_destroy(h: _Handle):
    if h is not None and h.ptr:
        lib().hw_destroy(h.ptr)
        h.ptr = None


def hw_init(h: _Handle, hh, hu, hv, b, deriv: Sequence):
    arrays = [hh, hu, hv, b, *deriv]
    kind = _kind(arrays)
    nd = 8 if h.grid.dim == 2 else 3
    if len(deriv) != nd:
        raise ValueError("deriv needs %d planes" % nd)
    P = _pp([_ptr(a, h.n) for a in deriv])
    _check(lib().hw_init(h.ptr, _ptr(hh, h.n), _ptr(hu, h.n), _ptr(hv, h.n) if hv is not None else None,
                         _ptr(b, h.n), P, kind), "hw_init")


def hw_rhs(h: _Handle, out: Sequence):
    kind = _kind(out)
    _check(lib().hw_rhs(h.ptr, _pp([_ptr(a, h.n, True) for a in out]), kind), "hw_rhs")


def hw_alpha(h: _Handle):
    a = (C.c_double * 2)()
    _check(lib().hw_alpha(h.ptr, a), "hw_alpha")
    return a[0], a[1]


def hw_cfl_dt(h: _Handle) -> float:
    dt = C.c_double()
    _check(lib().hw_cfl_dt(h.ptr, C.byref(dt)), "hw_cfl_dt")
    return dt.value


def hw_rk3_step(h: _Handle, dt: float):
    _check(lib().hw_rk3_step(h.ptr, float(dt)), "hw_rk3_step")


def hw_rk3_stage(h: _Handle, k: int, dt: float):
    _check(lib().hw_rk3_stage(h.ptr, int(k), float(dt)), "hw_rk3_stage")


def hw_advance(h: _Handle, nsteps: int, t_end: float = -1.0, use_graph: bool = True):
    t = C.c_double()
    n = C.c_int()
    _check(lib().hw_advance(h.ptr, int(nsteps), float(t_end), int(bool(use_graph)), C.byref(t), C.byref(n)),
           "hw_advance")
    return t.value, n.value


def hw_get_state(h: _Handle, out: Sequence, layout: int = HW_LAYOUT_PHYSICAL):
    kind = _kind(out)
    _check(lib().hw_get_state(h.ptr, _pp([_ptr(a, h.n, True) for a in out]), int(layout), kind), "hw_get_state")


def hw_set_state(h: _Handle, planes: Sequence, layout: int = HW_LAYOUT_PHYSICAL):
    kind = _kind(planes)
    _check(lib().hw_set_state(h.ptr, _pp([_ptr(a, h.n) for a in planes]), int(layout), kind), "hw_set_state")


def hw_get_base(h: _Handle, out: Sequence):
    kind = _kind(out)
    _check(lib().hw_get_base(h.ptr, _pp([_ptr(a, h.n, True) for a in out]), kind), "hw_get_base")


def hw_sync(h: _Handle):
    _check(lib().hw_sync(h.ptr), "hw_sync")


HW_PROF_NAMES = ["alpha", "sweep_x", "sweep_y", "node", "other"]


def hw_set_profiling(h: _Handle, on: bool):
    _check(lib().hw_set_profiling(h.ptr, int(bool(on))), "hw_set_profiling")


def hw_get_profile(h: _Handle):
    """{class: (ms, launches)} accumulated since the last call."""
    ms = (C.c_double * 5)()
    n = (C.c_int * 5)()
    _check(lib().hw_get_profile(h.ptr, ms, n), "hw_get_profile")
    return {k: (ms[i], n[i]) for i, k in enumerate(HW_PROF_NAMES)}


def hw_get_time(h: _Handle):
    """(simulated time, steps that advanced it)."""
    t, n = C.c_double(), C.c_longlong()
    _check(lib().hw_get_time(h.ptr, C.byref(t), C.byref(n)), "hw_get_time")
    return t.value, n.value


def hw_set_time(h: _Handle, t: float, steps: int):
    _check(lib().hw_set_time(h.ptr, float(t), int(steps)), "hw_set_time")


def hw_selftest_fp64_int(op: int, n: int, seed: int = 1):
    """Device check of the integer-pipe FP64 multiply (op 0, bitwise against DMUL), reciprocal (op 1,
    within one ulp of the correctly rounded one) or multiply by the kernels' literal constants (op 2,
    bitwise) on n operands: returns (accepted, mismatches, rejected operands that the fast path must
    take); the last two must be 0."""
    counts = (C.c_longlong * 3)()
    _check(lib().hw_selftest_fp64_int(int(op), int(n), int(seed), counts), "hw_selftest_fp64_int")
    return tuple(int(v) for v in counts)


def hw_measure_fp64_peak(reps: int = 5):
    """FP64 fma throughput of the current GPU: (best fma/s, median fma/s, best launch ms)."""
    out = (C.c_double * 3)()
    _check(lib().hw_measure_fp64_peak(int(reps), out), "hw_measure_fp64_peak")
    return out[0], out[1], out[2]


def hw_rhs1d_noalloc(grid: hw_grid, params: hw_params, hh, hu, b, deriv: Sequence, out: Sequence, stream=None):
    """Allocation-free 1D right-hand side; every plane is a CUDA tensor of grid.nx float64 values."""
    L = lib()
    f = L.hw_rhs1d_noalloc
    if f.argtypes is None:
        f.argtypes = [C.POINTER(hw_grid), C.POINTER(hw_params), C.c_void_p, C.c_void_p, C.c_void_p,
                      C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p]
        f.restype = C.c_int
    if _kind([hh, hu, b, *deriv, *out]) != HW_DEVICE:
        raise ValueError("hw_rhs1d_noalloc takes device tensors only")
    n = grid.nx
    _check(f(C.byref(grid), C.byref(params), _ptr(hh, n), _ptr(hu, n), _ptr(b, n), _pp([_ptr(a, n) for a in deriv]),
             _pp([_ptr(a, n, True) for a in out]), _stream_handle(stream)), "hw_rhs1d_noalloc")


# ------------------------------------------------------------------------------------------------
# block decomposition of one grid
# ------------------------------------------------------------------------------------------------
HW_FACE_W, HW_FACE_E, HW_FACE_S, HW_FACE_N = 0, 1, 2, 3
HW_HALO_NEIGHBOR, HW_HALO_MIRROR, HW_HALO_REPLICATE = 0, 1, 2


class hw_part_info(C.Structure):
    _fields_ = [("i0", C.c_int), ("j0", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("nbr", C.c_int * 4), ("mode", C.c_int * 4)]


def _dd_sigs():
    L = lib()
    if getattr(L, "_dd_ready", False):
        return L
    vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    pp = C.POINTER(C.c_void_p)
    for name, args in {
        "hw_dd_partition": [C.POINTER(hw_grid), i, i, i, C.POINTER(hw_part_info)],
        "hw_part_create": [C.POINTER(hw_grid), C.POINTER(hw_params), i, i, i, vp, C.POINTER(vp)],
        "hw_part_init": [vp, pp, ll, i],
        "hw_part_finish_init": [vp],
        "hw_halo_strip_size": [vp, i, i, C.POINTER(ll)],
        "hw_halo_pack": [vp, i, i, vp],
        "hw_halo_unpack": [vp, i, i, i, vp],
        "hw_part_alpha_keys": [vp, vp],
        "hw_part_stage": [vp, i, vp, d],
        "hw_dd_max_keys": [vp, i, vp, vp],
        "hw_dd_create": [C.POINTER(hw_grid), C.POINTER(hw_params), i, i, vp, C.POINTER(vp)],
        "hw_dd_init": [vp, vp, vp, vp, vp, pp, i],
        "hw_dd_advance": [vp, i, d, i, C.POINTER(d), C.POINTER(i)],
        "hw_dd_get_state": [vp, pp, i, i],
        "hw_dd_destroy": [vp],
        "hw_dd_adjoint_run": [vp, i, C.POINTER(d), C.POINTER(i), i, C.POINTER(d), C.POINTER(d), pp, pp],
        "hw_part_adj_create": [vp, i, i, i, C.POINTER(i), C.POINTER(i), i, C.POINTER(vp)],
        "hw_part_adj_destroy": [vp],
        "hw_part_adj_strip_size": [vp, i, i, C.POINTER(ll)],
        "hw_part_adj_pack": [vp, i, i, i, vp],
        "hw_part_adj_unpack": [vp, i, i, i, i, vp],
        "hw_part_adj_alpha_keys": [vp, i, i, vp],
        "hw_part_adj_forward_stage": [vp, i, i, d, vp],
        "hw_part_adj_gauges": [vp, C.POINTER(d)],
        "hw_part_adj_set_misfit": [vp, C.POINTER(d), C.POINTER(d), C.POINTER(d)],
        "hw_part_adj_reverse_stage": [vp, i, i, d, C.POINTER(d), C.POINTER(i)],
        "hw_part_adj_alpha_apply": [vp, C.POINTER(d), C.POINTER(i)],
        "hw_part_adj_rpack": [vp, i, i, vp],
        "hw_part_adj_radd": [vp, i, i, i, vp],
        "hw_part_adj_finish_static": [vp],
        "hw_part_adj_gradients": [vp, pp, pp, i, i],
    }.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = i
    L._dd_ready = True
    return L


def hw_dd_partition(grid: hw_grid, px: int, py: int, part: int) -> hw_part_info:
    """Block `part` of the grid split px x py (host only: no GPU needed)."""
    out = hw_part_info()
    _check(_dd_sigs().hw_dd_partition(C.byref(grid), int(px), int(py), int(part), C.byref(out)), "hw_dd_partition")
    return out


def _dev_ptr(t):
    if t is None or not _is_torch(t) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("a contiguous CUDA tensor is required")
    return C.c_void_p(t.data_ptr())


def hw_part_create(grid: hw_grid, params: hw_params, px: int, py: int, part: int, stream=None) -> _Handle:
    out = C.c_void_p()
    _check(_dd_sigs().hw_part_create(C.byref(grid), C.byref(params), int(px), int(py), int(part),
                                     _stream_handle(stream), C.byref(out)), "hw_part_create")
    info = hw_dd_partition(grid, px, py, part)
    ext = hw_grid(2, info.nx + 4, info.ny + 4, grid.x0, grid.x1, grid.y0, grid.y1, HW_BC_OUTFLOW, HW_BC_OUTFLOW)
    h = _Handle(out, ext, params, ext.nx * ext.ny, 9)
    h.info = info
    return h


def hw_part_init(h: _Handle, planes12: Sequence, ld: int):
    """planes12: the block's own nodes of h, hu, hv, b, h_x, hu_x, hv_x, h_y, hu_y, hv_y, b_x, b_y (numpy or
    CUDA, rows ld apart; each array's first element is the block's first node)."""
    kind = _kind(planes12)
    ptrs = []
    for a in planes12:
        if _is_torch(a):
            ptrs.append(_dev_ptr(a))
        else:
            if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host planes must be C-contiguous float64 numpy arrays")
            ptrs.append(C.c_void_p(a.ctypes.data))
    _check(_dd_sigs().hw_part_init(h.ptr, _pp(ptrs), int(ld), kind), "hw_part_init")


def hw_part_finish_init(h: _Handle):
    _check(_dd_sigs().hw_part_finish_init(h.ptr), "hw_part_finish_init")


class PartAdjoint:
    """The per-block adjoint context (hw_part_adj_*) of block solver `h` for a run of nsteps with the
    gauges of the global list that lie on the block's own nodes (slots and global node indices)."""

    def __init__(self, h: _Handle, nsteps: int, ngauge: int, slots: Sequence[int], nodes: Sequence[int], global_nx: int):
        L = _dd_sigs()
        n = len(slots)
        sl = (C.c_int * max(n, 1))(*[int(x) for x in slots])
        nd = (C.c_int * max(n, 1))(*[int(x) for x in nodes])
        out = C.c_void_p()
        _check(L.hw_part_adj_create(h.ptr, int(nsteps), int(ngauge), n, sl, nd, int(global_nx), C.byref(out)),
               "hw_part_adj_create")
        self.ptr, self.h, self.nsteps, self.ngauge = out, h, nsteps, ngauge

    def close(self):
        if self.ptr:
            _dd_sigs().hw_part_adj_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def strip_size(self, what: int, face: int) -> int:
        n = C.c_longlong()
        _check(_dd_sigs().hw_part_adj_strip_size(self.ptr, int(what), int(face), C.byref(n)), "hw_part_adj_strip_size")
        return n.value

    def pack(self, j: int, k: int, face: int, strip):
        _check(_dd_sigs().hw_part_adj_pack(self.ptr, int(j), int(k), int(face), _dev_ptr(strip)), "hw_part_adj_pack")

    def unpack(self, j: int, k: int, face: int, mode: int, strip):
        _check(_dd_sigs().hw_part_adj_unpack(self.ptr, int(j), int(k), int(face), int(mode), _dev_ptr(strip)),
               "hw_part_adj_unpack")

    def alpha_keys(self, j: int, k: int, keys):
        _check(_dd_sigs().hw_part_adj_alpha_keys(self.ptr, int(j), int(k), _dev_ptr(keys)), "hw_part_adj_alpha_keys")

    def forward_stage(self, j: int, k: int, dt: float, keys):
        _check(_dd_sigs().hw_part_adj_forward_stage(self.ptr, int(j), int(k), float(dt), _dev_ptr(keys)),
               "hw_part_adj_forward_stage")

    def gauges(self) -> np.ndarray:
        out = np.zeros(self.nsteps * self.ngauge)
        _check(_dd_sigs().hw_part_adj_gauges(self.ptr, out.ctypes.data_as(C.POINTER(C.c_double))), "hw_part_adj_gauges")
        return out

    def set_misfit(self, gvals, obs) -> float:
        """Starts the reverse pass; returns the loss (summed as the library's other adjoint entry points)."""
        g = np.ascontiguousarray(gvals, dtype=np.float64).ravel()
        o = np.ascontiguousarray(obs, dtype=np.float64).ravel()
        if g.size != self.nsteps * self.ngauge or o.size != g.size:
            raise ValueError("gauge values and observations need nsteps x ngauge entries")
        D = C.POINTER(C.c_double)
        loss = C.c_double()
        _check(_dd_sigs().hw_part_adj_set_misfit(self.ptr, g.ctypes.data_as(D), o.ctypes.data_as(D), C.byref(loss)),
               "hw_part_adj_set_misfit")
        return loss.value

    def reverse_stage(self, j: int, k: int, dt: float):
        """(alpha adjoint share [2], first maximising global nodes [2])."""
        la = (C.c_double * 2)()
        am = (C.c_int * 2)()
        _check(_dd_sigs().hw_part_adj_reverse_stage(self.ptr, int(j), int(k), float(dt), la, am),
               "hw_part_adj_reverse_stage")
        return [la[0], la[1]], [am[0], am[1]]

    def alpha_apply(self, lalpha, argmax):
        la = (C.c_double * 2)(*[float(x) for x in lalpha])
        am = (C.c_int * 2)(*[int(x) for x in argmax])
        _check(_dd_sigs().hw_part_adj_alpha_apply(self.ptr, la, am), "hw_part_adj_alpha_apply")

    def rpack(self, what: int, face: int, strip):
        _check(_dd_sigs().hw_part_adj_rpack(self.ptr, int(what), int(face), _dev_ptr(strip)), "hw_part_adj_rpack")

    def radd(self, what: int, face: int, mode: int, strip):
        _check(_dd_sigs().hw_part_adj_radd(self.ptr, int(what), int(face), int(mode), _dev_ptr(strip)),
               "hw_part_adj_radd")

    def finish_static(self):
        _check(_dd_sigs().hw_part_adj_finish_static(self.ptr), "hw_part_adj_finish_static")

    def gradients(self):
        """The block's own nodes of the state gradient (9 planes) and the static one (3), host arrays."""
        info = self.h.info
        gs = [np.empty((info.ny, info.nx)) for _ in range(9)]
        gb = [np.empty((info.ny, info.nx)) for _ in range(3)]
        _check(_dd_sigs().hw_part_adj_gradients(self.ptr, _pp([C.c_void_p(a.ctypes.data) for a in gs]),
                                                 _pp([C.c_void_p(a.ctypes.data) for a in gb]), info.nx, HW_HOST),
               "hw_part_adj_gradients")
        return gs, gb


def hw_halo_strip_size(h: _Handle, set_: int, face: int) -> int:
    n = C.c_longlong()
    _check(_dd_sigs().hw_halo_strip_size(h.ptr, int(set_), int(face), C.byref(n)), "hw_halo_strip_size")
    return n.value


def hw_halo_pack(h: _Handle, set_: int, face: int, strip):
    _check(_dd_sigs().hw_halo_pack(h.ptr, int(set_), int(face), _dev_ptr(strip)), "hw_halo_pack")


def hw_halo_unpack(h: _Handle, set_: int, face: int, mode: int, strip):
    _check(_dd_sigs().hw_halo_unpack(h.ptr, int(set_), int(face), int(mode), _dev_ptr(strip)), "hw_halo_unpack")


def hw_part_alpha_keys(h: _Handle, keys):
    _check(_dd_sigs().hw_part_alpha_keys(h.ptr, _dev_ptr(keys)), "hw_part_alpha_keys")


def hw_part_stage(h: _Handle, k: int, keys, t_end: float = -1.0):
    _check(_dd_sigs().hw_part_stage(h.ptr, int(k), _dev_ptr(keys), float(t_end)), "hw_part_stage")


def hw_dd_max_keys(keys, out, stream=None):
    """out (2 int64, CUDA) = maxima over the rows of keys (n x 2 int64, CUDA)."""
    n = keys.numel() // 2
    _check(_dd_sigs().hw_dd_max_keys(_dev_ptr(keys), int(n), _dev_ptr(out), _stream_handle(stream)), "hw_dd_max_keys")


class _DDHandle:
    def __init__(self, ptr, grid):
        self.ptr, self.grid = ptr, grid


def hw_dd_create(grid: hw_grid, params: hw_params, px: int, py: int, stream=None) -> _DDHandle:
    out = C.c_void_p()
    _check(_dd_sigs().hw_dd_create(C.byref(grid), C.byref(params), int(px), int(py), _stream_handle(stream),
                                   C.byref(out)), "hw_dd_create")
    return _DDHandle(out, grid)


def hw_dd_destroy(d: _DDHandle):
    if d is not None and d.ptr:
        _dd_sigs().hw_dd_destroy(d.ptr)
        d.ptr = None


def hw_dd_init(d: _DDHandle, hh, hu, hv, b, deriv: Sequence):
    n = d.grid.nx * d.grid.ny
    kind = _kind([hh, hu, hv, b, *deriv])
    _check(_dd_sigs().hw_dd_init(d.ptr, _ptr(hh, n), _ptr(hu, n), _ptr(hv, n), _ptr(b, n),
                                 _pp([_ptr(a, n) for a in deriv]), kind), "hw_dd_init")


def hw_dd_advance(d: _DDHandle, nsteps: int, t_end: float = -1.0, use_graph: bool = True):
    t, n = C.c_double(), C.c_int()
    _check(_dd_sigs().hw_dd_advance(d.ptr, int(nsteps), float(t_end), int(bool(use_graph)), C.byref(t), C.byref(n)),
           "hw_dd_advance")
    return t.value, n.value


def hw_dd_get_state(d: _DDHandle, out: Sequence, layout: int = HW_LAYOUT_EQUILIBRIUM):
    n = d.grid.nx * d.grid.ny
    _check(_dd_sigs().hw_dd_get_state(d.ptr, _pp([_ptr(a, n, True) for a in out]), int(layout), _kind(out)),
           "hw_dd_get_state")


def hw_dd_adjoint_run(d: _DDHandle, dts, gauge_idx, eta_obs, grad_state: Sequence, grad_static: Sequence):
    """Gauge misfit and its gradient over the blocks (whole-run tape); gradients are CUDA tensors of the
    global grid. Returns the loss."""
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    gi = np.ascontiguousarray(gauge_idx, dtype=np.int32)
    ob = np.ascontiguousarray(eta_obs, dtype=np.float64)
    n = d.grid.nx * d.grid.ny
    loss = C.c_double()
    _check(_dd_sigs().hw_dd_adjoint_run(d.ptr, len(dts), dts.ctypes.data_as(C.POINTER(C.c_double)),
                                        gi.ctypes.data_as(C.POINTER(C.c_int)), len(gi),
                                        ob.ctypes.data_as(C.POINTER(C.c_double)), C.byref(loss),
                                        _pp([_ptr(a, n, True) for a in grad_state]),
                                        _pp([_ptr(a, n, True) for a in grad_static])), "hw_dd_adjoint_run")
    return loss.value


class DecomposedSolver:
    """One 2D grid split into px x py blocks on the current GPU (halo exchange between them on the device);
    the same results as ``Solver``, bit for bit."""

    def __init__(self, sc, px: int, py: int, params: Optional[hw_params] = None, stream=None):
        self.grid = make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y, dim=2)
        self.params = params or make_params(eps_w=sc.eps_w)
        self.h = hw_dd_create(self.grid, self.params, px, py, stream)
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in [sc.h, sc.hu, sc.hv, sc.b] + list(sc.deriv)]
        hw_dd_init(self.h, arrs[0], arrs[1], arrs[2], arrs[3], arrs[4:])

    def close(self):
        hw_dd_destroy(self.h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def advance(self, nsteps, t_end=-1.0, use_graph=True):
        return hw_dd_advance(self.h, nsteps, t_end, use_graph)

    def state(self, layout=HW_LAYOUT_EQUILIBRIUM):
        out = [np.empty((self.grid.ny, self.grid.nx)) for _ in range(9)]
        hw_dd_get_state(self.h, out, layout)
        return out


# ------------------------------------------------------------------------------------------------
# batched form
# ------------------------------------------------------------------------------------------------
def _batch_sigs():
    L = lib()
    if getattr(L, "_batch_ready", False):
        return L
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    pp = C.POINTER(C.c_void_p)
    for name, args in {
        "hw_batch_create": [i, C.POINTER(hw_grid), C.POINTER(hw_params), vp, C.POINTER(vp)],
        "hw_batch_destroy": [vp],
        "hw_batch_init": [vp, i, vp, vp, vp, vp, pp, i],
        "hw_batch_run": [vp, i, i],
        "hw_batch_get_state": [vp, i, pp, i, i],
        "hw_batch_get_time": [vp, C.POINTER(d), C.POINTER(i)],
        "hw_batch_set_tiles": [vp, i, i],
        "hw_batch_get_tiles": [vp, i, C.POINTER(i)],
        "hw_batch_time_tiles": [vp, i, C.POINTER(i), i, i, C.POINTER(d), C.POINTER(d)],
        "hw_batch_set_persistent": [vp, i],
        "hw_batch_get_persistent": [vp, C.POINTER(i), C.POINTER(i)],
        "hw_batch_test_barrier_timeout": [vp],
        "hw_batch_get_phase_times": [vp, C.POINTER(d)],
    }.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = i
    L._batch_ready = True
    return L


class _BHandle:
    def __init__(self, ptr, grids):
        self.ptr, self.grids = ptr, grids


def hw_batch_create(grids: Sequence[hw_grid], params: hw_params, stream=None) -> _BHandle:
    L = _batch_sigs()
    arr = (hw_grid * len(grids))(*grids)
    out = C.c_void_p()
    _check(L.hw_batch_create(len(grids), arr, C.byref(params), _stream_handle(stream), C.byref(out)), "hw_batch_create")
    return _BHandle(out, list(grids))


def hw_batch_destroy(b: _BHandle):
    if b is not None and b.ptr:
        _batch_sigs().hw_batch_destroy(b.ptr)
        b.ptr = None


def hw_batch_init(b: _BHandle, i: int, hh, hu, hv, bb, deriv: Sequence):
    g = b.grids[i]
    n = g.nx * g.ny
    kind = _kind([hh, hu, hv, bb, *deriv])
    _check(_batch_sigs().hw_batch_init(b.ptr, i, _ptr(hh, n), _ptr(hu, n), _ptr(hv, n), _ptr(bb, n),
                                       _pp([_ptr(a, n) for a in deriv]), kind), "hw_batch_init")


def hw_batch_run(b: _BHandle, nsteps: int, use_graph: bool = True):
    _check(_batch_sigs().hw_batch_run(b.ptr, int(nsteps), int(bool(use_graph))), "hw_batch_run")


def hw_batch_get_state(b: _BHandle, i: int, out: Sequence, layout: int = HW_LAYOUT_EQUILIBRIUM):
    g = b.grids[i]
    n = g.nx * g.ny
    _check(_batch_sigs().hw_batch_get_state(b.ptr, i, _pp([_ptr(a, n, True) for a in out]), int(layout), _kind(out)),
           "hw_batch_get_state")


def hw_batch_get_time(b: _BHandle):
    n = len(b.grids)
    t = (C.c_double * n)()
    k = (C.c_int * n)()
    _check(_batch_sigs().hw_batch_get_time(b.ptr, t, k), "hw_batch_get_time")
    return np.array(t[:]), np.array(k[:])


def hw_batch_set_tiles(b: _BHandle, i: int, yc: int):
    """y-tile width of grid i: 1, 2 or 4 columns per tile."""
    _check(_batch_sigs().hw_batch_set_tiles(b.ptr, int(i), int(yc)), "hw_batch_set_tiles")


def hw_batch_get_tiles(b: _BHandle, i: int) -> int:
    yc = C.c_int()
    _check(_batch_sigs().hw_batch_get_tiles(b.ptr, int(i), C.byref(yc)), "hw_batch_get_tiles")
    return yc.value


def hw_batch_time_tiles(b: _BHandle, ids: Sequence[int], yc: int, reps: int = 3):
    arr = (C.c_int * len(ids))(*[int(i) for i in ids])
    mx, my = C.c_double(), C.c_double()
    _check(_batch_sigs().hw_batch_time_tiles(b.ptr, len(ids), arr, int(yc), int(reps), C.byref(mx), C.byref(my)),
           "hw_batch_time_tiles")
    return mx.value, my.value


def hw_batch_set_persistent(b: _BHandle, on: bool):
    """on: one cooperative launch per step (phases separated by bounded grid barriers); off: one launch per
    phase (the default)."""
    _check(_batch_sigs().hw_batch_set_persistent(b.ptr, int(bool(on))), "hw_batch_set_persistent")


def hw_batch_get_persistent(b: _BHandle):
    """(on, blocks): the launch form and the persistent step kernel's block count."""
    on, blocks = C.c_int(), C.c_int()
    _check(_batch_sigs().hw_batch_get_persistent(b.ptr, C.byref(on), C.byref(blocks)), "hw_batch_get_persistent")
    return bool(on.value), blocks.value


def hw_batch_test_barrier_timeout(b: _BHandle) -> int:
    """One persistent step launch in which block 0 never reaches the first grid barrier (2 ms bound); returns
    the C code: HW_ERR_TIMEOUT (-5) when the bounded wait worked."""
    return int(_batch_sigs().hw_batch_test_barrier_timeout(b.ptr))


BSTEP_PHASE_NAMES = [f"stage{k}_{p}" for k in (1, 2, 3) for p in ("alpha_coarse", "alpha_exact", "alpha_dt",
                                                                   "sweeps", "node")]


def hw_batch_get_phase_times(b: _BHandle) -> dict:
    """Phase durations (ms) of the last persistent step launch, keyed by BSTEP_PHASE_NAMES."""
    ms = (C.c_double * 15)()
    _check(_batch_sigs().hw_batch_get_phase_times(b.ptr, ms), "hw_batch_get_phase_times")
    return dict(zip(BSTEP_PHASE_NAMES, ms[:]))


class BatchedSolver:
    """Many 2D grids advancing together, with a CUDA graph of two steps: one launch per phase over all grids
    (persistent=False), or one cooperative launch per step (persistent=True)."""

    def __init__(self, scenarios, params: Optional[hw_params] = None, stream=None, persistent: bool = False):
        grids = [make_grid(s.nx, s.ny, s.x0, s.x1, s.y0, s.y1, s.bc_x, s.bc_y, dim=2) for s in scenarios]
        self.params = params or make_params()
        self.h = hw_batch_create(grids, self.params, stream)
        self.grids = grids
        for i, s in enumerate(scenarios):
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in [s.h, s.hu, s.hv, s.b] + list(s.deriv)]
            hw_batch_init(self.h, i, arrs[0], arrs[1], arrs[2], arrs[3], arrs[4:])
        if persistent:
            hw_batch_set_persistent(self.h, True)

    def set_persistent(self, on: bool):
        hw_batch_set_persistent(self.h, on)

    @property
    def persistent(self):
        return hw_batch_get_persistent(self.h)[0]

    def close(self):
        hw_batch_destroy(self.h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, nsteps, use_graph=True):
        hw_batch_run(self.h, nsteps, use_graph)

    def state(self, i, layout=HW_LAYOUT_EQUILIBRIUM):
        g = self.grids[i]
        out = [np.empty((g.ny, g.nx)) for _ in range(9)]
        hw_batch_get_state(self.h, i, out, layout)
        return out

    def times(self):
        return hw_batch_get_time(self.h)

    def autotune(self, cache_path: Optional[str] = None, reps: int = 3):
        from . import autotune
        return autotune.tune(self, cache_path=cache_path, reps=reps)


def hw_version() -> str:
    return lib().hw_version().decode()


# ------------------------------------------------------------------------------------------------
# convenience object over the C names
# ------------------------------------------------------------------------------------------------
class Solver:
    """One grid on the current CUDA device, bound to torch's current stream (or `stream`)."""

    def __init__(self, grid: hw_grid, params: hw_params, stream=None):
        self.h = hw_create(grid, params, stream)
        self.grid, self.params = grid, params
        self.shape = (grid.ny, grid.nx) if grid.dim == 2 else (grid.nx,)

    def close(self):
        hw_destroy(self.h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @classmethod
    def from_scenario(cls, sc, params: Optional[hw_params] = None, stream=None, device: bool = False):
        """Create and initialise from a ``scenarios.Scenario`` (host arrays, or copied to the GPU)."""
        grid = make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y, dim=sc.dim)
        if params is None:
            params = make_params(eps_w=sc.eps_w)
        s = cls(grid, params, stream)
        arrs = [sc.h, sc.hu, sc.hv if sc.dim == 2 else None, sc.b] + list(sc.deriv)
        if device:
            import torch
            arrs = [None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
                    for a in arrs]
        else:
            arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
        hw_init(s.h, arrs[0], arrs[1], arrs[2], arrs[3], arrs[4:])
        return s

    def _planes(self, count):
        return [np.empty(self.shape) for _ in range(count)]

    def rhs(self):
        out = self._planes(self.h.nstate)
        hw_rhs(self.h, out)
        return out

    def alpha(self):
        return hw_alpha(self.h)

    def cfl_dt(self):
        return hw_cfl_dt(self.h)

    def rk3_step(self, dt):
        hw_rk3_step(self.h, dt)

    def rk3_stage(self, k, dt):
        hw_rk3_stage(self.h, k, dt)

    def advance(self, nsteps, t_end=-1.0, use_graph=True):
        return hw_advance(self.h, nsteps, t_end, use_graph)

    def state(self, layout=HW_LAYOUT_EQUILIBRIUM):
        out = self._planes(self.h.nstate)
        hw_get_state(self.h, out, layout)
        return out

    def set_state(self, planes, layout=HW_LAYOUT_EQUILIBRIUM):
        hw_set_state(self.h, [np.ascontiguousarray(p, dtype=np.float64) for p in planes], layout)

    def base(self):
        out = self._planes(self.h.nstate)
        hw_get_base(self.h, out)
        return out

    def sync(self):
        hw_sync(self.h)
