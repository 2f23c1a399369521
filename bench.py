#!/usr/bin/env python
"""Benchmark of the 2D well-balanced fifth-order FD HWENO scheme on GB300.

Workload: 2048 x 2048 nodes on [0,2] x [0,1], reflective walls, seeded bottom of 8 Gaussian bumps,
still water eta = 1 plus a 0.01 strip on x in [0.05, 0.15], state = 3 conserved variables and their
x and y derivatives, SSP-RK3 at CFL 0.6 with the time step computed on the device.
A step is one SSP-RK3 step (3 stages) over the whole grid. Metric: FP64 point-updates/s
(grid points x RK stages per second), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the CPU oracle (the plain FP64 restatement of the paper's scheme used by the
tests) on this machine's host cores on the same workload. Multi-GPU runs are independent replicas
of the workload (one per rank, no data exchange), so `value` scales weakly.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 2048
STAGES = 3
WORKLOAD = ("2D plain scheme, 2048x2048 on [0,2]x[0,1], reflective walls, 8 Gaussian bumps (seeded), "
            "eta=1 + 0.01 strip on x in [0.05,0.15], SSP-RK3 CFL 0.6, dt on device")
METRIC = "FP64 point-updates/s (grid pts x RK stages) at 2048^2"
UNIT = "point-updates/s"

# Algorithmic FP64 work per unit of each kernel, tallied from the formulas the kernels evaluate
# (the design notes list every term): "ops" counts add, mul and fma as one FP64 operation each,
# "flops" counts an fma as 2. A reciprocal is a hardware seed plus three fma, a reciprocal square
# root a seed plus five operations. Sweeps: 432 operations per interface plus about 1.03 node
# records of 42 operations; node kernel averaged over the three RK stages.
ALGO = {
    "sweep_x": {"ops": 475.0, "flops": 685.7},  # per x-interface
    "sweep_y": {"ops": 475.7, "flops": 686.7},  # per y-interface
    "node": {"ops": 365.0, "flops": 511.0},     # per node
    "alpha": {"ops": 15.0, "flops": 27.0},      # per node
}
UNITS_PER_LAUNCH = {
    "sweep_x": (NX + 1) * NY,
    "sweep_y": NX * (NY + 1),
    "node": NX * NY,
    "alpha": NX * NY,
}
# FP64 peak: measured live on the benchmark's GPU (hw_measure_fp64_peak, independent fma chains on every
# SM, median of 20 launches). The nominal figure from the unit counts and the clock (152 SMs x 2 DFMA per
# SM per cycle, the FP64 pipe peak ncu reports on GB300, x 2 flops x 2.07 GHz) is kept for comparison.
SMS, DFMA_PER_SM_CLK, SM_GHZ = 152, 2, 2.07
NOMINAL_FP64_TFLOPS = SMS * DFMA_PER_SM_CLK * 2 * SM_GHZ / 1e3
PEAK_FP64_TFLOPS = NOMINAL_FP64_TFLOPS  # replaced by the measured figure in main()
PEAK_FP64_OPS = SMS * DFMA_PER_SM_CLK * SM_GHZ * 1e9
# Algorithmic DRAM bytes of one RK stage per node, the minimum a fused stage must move: stage 1 reads the
# 9 state and 3 static planes and writes 9 state and 6 limited-derivative planes; stages 2 and 3 read the
# 9 state, 3 static and 9 base planes and write 9 (limiter recomputed: 27 planes of 8 bytes on average).
# The whole-step HBM fraction is taken against it.
ALGO_BYTES_PER_NODE_STAGE = 216.0
# DRAM bytes per unit from ncu captures (dram__bytes_read.sum + dram__bytes_write.sum of one launch of this
# benchmark at 2048^2, a one-pass capture; the node kernel at RK stage 3), valid only for the kernel sources
# they were taken on (sources_sha); times the units of a launch.
TRAFFIC = {
    "sweep_x": {"bytes_per_unit": 231.5, "sha": "e0ac982961c54e0f"},
    "sweep_y": {"bytes_per_unit": 235.4, "sha": "e0ac982961c54e0f"},
    "node": {"bytes_per_unit": 533.9, "sha": "e0ac982961c54e0f"},
}
# FP64-pipe instructions per unit (ncu --set full at 2048x1024: DFMA + DADD + DMUL thread instructions of
# one launch over its units; the count per unit does not depend on the grid size). Part of the products
# run on the integer pipes (each bit-identical to DMUL), so these are below the algorithmic "ops" above;
# valid only for the kernel sources they were taken on (sources_sha).
FP64_PIPE_OPS = {
    "sweep_x": {"ops_per_unit": 341.9, "sha": "e0ac982961c54e0f"},
    "sweep_y": {"ops_per_unit": 342.8, "sha": "e0ac982961c54e0f"},
    "node": {"ops_per_unit": 243.0, "sha": "e0ac982961c54e0f"},
}
STATE_BYTES = 9 * NX * NY * 8


def hbm_peak():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


FORWARD_SOURCES = ("hw_device.cuh", "hw_fp64_int.h", "hw_stencil2d.cuh", "hw_kernels2d.cu", "hw_internal.h")


def sources_sha():
    """sha256 (16 hex digits) of the code the timed 2D kernels are compiled from (line comments and
    blank lines left out, so that editing a comment does not invalidate a capture)."""
    import hashlib
    import re
    d = os.path.join(ROOT, "paper_2208_01260_gb300", "csrc")
    h = hashlib.sha256()
    for f in FORWARD_SOURCES:
        for ln in open(os.path.join(d, f)).read().splitlines():
            code = re.sub(r"//.*$", "", ln).rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(backend="nccl"):
    """Rank layout from the launcher's environment; a process group only when WORLD_SIZE > 1."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return ws, rank, local


def _reduce(x, ws, op):
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def allreduce_max(x, ws):
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.MAX if ws > 1 else None)


def allreduce_sum(x, ws):
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.SUM if ws > 1 else None)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def job_rate(units_local, seconds_local, ws):
    """Whole-job throughput: every rank's units over the slowest rank's time (each rank advances its own
    replica; no data-path collective). Returns (units/s, max seconds, total units)."""
    seconds = allreduce_max(seconds_local, ws)
    units = allreduce_sum(units_local, ws)
    return units / seconds, seconds, units


def oracle_rate(seconds_budget=60.0):
    """Oracle (CPU, all host cores) on the same workload: one RK3 step of the full 2048^2 grid if it fits
    the budget, else the first stage only. Returns (point-updates/s, sample description, threads)."""
    import oracle
    from paper_2208_01260_gb300 import scenarios as S
    sc = S.bumps2d(NX, NY, strip=0.01)
    g = oracle.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y)
    p = oracle.make_params()
    st, stat = oracle.to_state2d(sc.h, sc.hu, sc.hv, sc.b, sc.deriv)
    dt = oracle.cfl_dt2d(g, p, st, stat)
    t0 = time.perf_counter()
    out, base, _ = oracle.stage2d(g, p, 1, dt, st, stat)
    t1 = time.perf_counter()
    stages, elapsed = 1, t1 - t0
    if 3 * elapsed < seconds_budget:
        out2, _, _ = oracle.stage2d(g, p, 2, dt, out, stat, base)
        oracle.stage2d(g, p, 3, dt, out2, stat, base)
        stages, elapsed = 3, time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = "%d RK stage(s) of the full 2048x2048 workload" % stages
    return NX * NY * stages / elapsed, desc, threads, elapsed


ONEDIM_RUNS = (("config1_n200_t0.2", "perturbed1d", 0.2), ("ex41_n1600_t0.1", "accuracy1d", 0.1))


def _onedim_scenario(kind):
    from paper_2208_01260_gb300 import scenarios as S
    return S.perturbed1d() if kind == "perturbed1d" else S.accuracy1d(1600)


def onedim(reps=5):
    """The 1D scheme (Sec. 2.1-2.2) on the paper's 1D grid sizes: config 1 (N = 200, reflective, two bumps,
    the 1e-3 pulse, epsilon 1e-10, CFL 0.6 to t = 0.2) and the accuracy sweep's largest grid (N = 1600,
    periodic, Ex. 4.1 data, CFL steps to t = 0.1). Each run goes from the initial state to t_end through
    hw_advance from its CUDA graph; host wall time around the call (it returns when the run is done),
    median of `reps` runs after one untimed run. Grids of a few hundred nodes leave the GPU launch-bound."""
    import torch
    import paper_2208_01260_gb300 as hw
    out = {}
    for name, kind, t_end in ONEDIM_RUNS:
        sc = _onedim_scenario(kind)
        s = hw.Solver.from_scenario(sc, hw.make_params(eps_w=sc.eps_w))
        st0 = s.state()
        times = []
        for r in range(reps + 1):
            hw.hw_set_state(s.h, st0, hw.HW_LAYOUT_EQUILIBRIUM)
            hw.hw_set_time(s.h, 0.0, 0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            t, n = s.advance(10 ** 6, t_end=t_end)
            el = time.perf_counter() - t0
            if r:
                times.append(el)
        s.close()
        el = statistics.median(times)
        out[name] = {"nx": sc.nx, "steps": n, "t_end": t, "run_ms": el * 1e3, "ms_per_step": el * 1e3 / n,
                     "value": sc.nx * STAGES * n / el, "unit": UNIT}
    out["how"] = ("whole run from the initial state to t_end through hw_advance (CUDA graph of two steps), host "
                  "wall time, median of %d runs" % reps)
    return out


def oracle_onedim():
    """The oracle on the runs of onedim(), one host core each (a 1D grid is one row: one OpenMP thread)."""
    import oracle
    out = {}
    for name, kind, t_end in ONEDIM_RUNS:
        sc = _onedim_scenario(kind)
        g = oracle.make_grid(sc.nx, 1, sc.x0, sc.x1, bc_x=sc.bc_x)
        p = oracle.make_params(eps_w=sc.eps_w)
        st, stat = oracle.to_state1d(sc.h, sc.hu, sc.b, sc.deriv)
        t0 = time.perf_counter()
        _, t, n = oracle.run1d(g, p, st, stat, t_end)
        el = time.perf_counter() - t0
        out[name] = {"nx": sc.nx, "steps": n, "run_ms": el * 1e3, "value": sc.nx * STAGES * n / el, "unit": UNIT,
                     "cores": 1}
    return out


def batched_compare(steps, n_inst=512, fixed=None):
    """Config 4: n_inst grids with nx, ny log-uniform in [64, 1024] (or all of size `fixed`) on
    [0,1]^2, reflective, seeded bathymetry and surface hump, each at its own CFL dt. Aggregate
    point-updates/s of the batched form (one launch per phase over all grids, CUDA graph; then the same
    batch with one cooperative launch per step) and of the plain loop (one single-grid solver per instance advanced one step at a time: with the library's
    cfl_dt() and rk3_step(dt), and, as a stronger baseline, with the device-side dt of hw_advance)."""
    import torch
    import paper_2208_01260_gb300 as hw
    from paper_2208_01260_gb300 import scenarios as S
    if fixed:
        nxs, nys = np.full(n_inst, fixed[0]), np.full(n_inst, fixed[1])
    else:
        nxs, nys = S.batch_sizes(n_inst)
    scs = [S.batch_scenario(i, int(nxs[i]), int(nys[i])) for i in range(n_inst)]
    pts = float(sum(int(a) * int(b) for a, b in zip(nxs, nys)))
    stream = torch.cuda.current_stream()
    b = hw.BatchedSolver(scs)
    tune = b.autotune()
    b.run(3, use_graph=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.run(steps, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    # the same batch (same tiles, states carried on) with one cooperative launch per step
    b.set_persistent(True)
    b.run(4, use_graph=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b.run(steps, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1)
    blocks = hw.hw_batch_get_persistent(b.h)[1]
    ph = hw.hw_batch_get_phase_times(b.h)  # the last timed step, per stage
    phases = {name: sum(ph["stage%d_%s" % (k, name)] for k in (1, 2, 3)) / 3
              for name in ("alpha_coarse", "alpha_exact", "alpha_dt", "sweeps", "node")}
    b.close()
    solvers = [hw.Solver.from_scenario(sc, hw.make_params()) for sc in scs]

    def plain_api_step(s):  # the library's own calls: cfl_dt() then rk3_step(dt)
        s.rk3_step(s.cfl_dt())

    def plain_device_dt_step(s):  # dt computed and applied on the device, no host round trip
        s.advance(1, use_graph=False)

    ms = {}
    for name, fn in (("api", plain_api_step), ("device_dt", plain_device_dt_step)):
        for s in solvers:
            fn(s)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            for s in solvers:
                fn(s)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[name] = e0.elapsed_time(e1)
    for s in solvers:
        s.close()
    vb = pts * STAGES * steps / (ms_b * 1e-3)
    vpers = pts * STAGES * steps / (ms_p * 1e-3)
    vp = pts * STAGES * steps / (ms["api"] * 1e-3)
    vd = pts * STAGES * steps / (ms["device_dt"] * 1e-3)
    return {"instances": n_inst, "total_points": int(pts), "steps": steps, "value_batched": vb, "value_plain": vp,
            "ratio": vb / vp, "ms_per_step_batched": ms_b / steps, "ms_per_step_plain": ms["api"] / steps,
            "plain": "per instance per step: cfl_dt() then rk3_step(dt)",
            "value_plain_device_dt": vd, "ratio_vs_device_dt_loop": vb / vd,
            "ms_per_step_plain_device_dt": ms["device_dt"] / steps,
            "plain_device_dt": "per instance per step: hw_advance(1 step), dt found and applied on the device",
            "value_batched_persistent": vpers, "ratio_persistent": vpers / vp,
            "ms_per_step_batched_persistent": ms_p / steps,
            "persistent_phase_ms_per_stage": phases,
            "persistent": "one cooperative launch of %d blocks per step, phases separated by grid barriers "
                          "(value_batched: 12 launches per step, one per phase)" % blocks,
            "unit": UNIT, "tiles": "autotuned per size class"}


# Algorithmic DRAM bytes per unit in single precision (4-byte planes): a sweep reads each node's 12
# state/static values and the interface's 6 source candidates and writes 12 interface values (30 planes);
# the node kernel reads 9 state, 3 static, 24 interface, 4 static-source and (stages 2-3) 9 base planes
# and writes 9 state and (stage 1) 9 base planes, 58 planes on average over the three stages; alpha reads
# eta, m, w, b.
ALGO_BYTES_FP32 = {"sweep_x": 30 * 4, "sweep_y": 30 * 4, "node": 58 * 4, "alpha": 4 * 4}


def fp32_variant(steps, warmup=3):
    """The same 2048^2 workload in single precision (the paper's single-precision runs): rate from the
    captured graph, and per kernel the algorithmic bytes over its event-timed duration against HBM."""
    import torch
    import paper_2208_01260_gb300 as hw
    from paper_2208_01260_gb300 import scenarios as S
    sc = S.bumps2d(NX, NY, strip=0.01)
    s = hw.Solver.from_scenario(sc, hw.make_params(precision=hw.HW_FP32))
    stream = torch.cuda.current_stream()
    s.advance(warmup, use_graph=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.advance(steps, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    hw.hw_set_profiling(s.h, True)
    s.advance(steps, use_graph=False)
    torch.cuda.synchronize()
    prof = hw.hw_get_profile(s.h)
    hw.hw_set_profiling(s.h, False)
    hbm, _ = hbm_peak()
    kernels = {}
    for k in ("sweep_x", "sweep_y", "node", "alpha"):
        tot, n = prof[k]
        if n == 0:
            continue
        nl = n if k != "alpha" else prof["sweep_x"][1]
        avg_s = tot / nl * 1e-3
        gbs = ALGO_BYTES_FP32[k] * UNITS_PER_LAUNCH[k] / avg_s / 1e9
        kernels[k] = {"ms_avg": avg_s * 1e3, "algorithmic_gbs": gbs, "hbm_frac": gbs / hbm}
    s.close()
    return {"value": NX * NY * STAGES * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "steps": steps, "dtype": "f32", "kernels": kernels, "hbm_peak_gbs": hbm,
            "note": "single-precision variant of the same workload (well-balance to float round-off); "
                    "not the headline, which is FP64"}


def adjoint_cost(n=512, nsteps=400, snapshots=20):
    """Config 5: gauge misfit over 32 gauges and `nsteps` steps at n x n (bottom of the benchmark plus
    a surface hump, reflective; observations from a run with another hump; the unperturbed CFL step
    sequence passed explicitly). Times the forward loss and the adjoint run, once on a whole-run tape
    and once with binomial checkpointing (`snapshots` states)."""
    import torch
    import paper_2208_01260_gb300 as hw
    from paper_2208_01260_gb300 import adjoint as A
    from paper_2208_01260_gb300 import scenarios as S

    def eq(sc):
        st = [sc.h + sc.b, sc.hu, sc.hv, sc.deriv[0] + sc.deriv[6], sc.deriv[1], sc.deriv[2],
              sc.deriv[3] + sc.deriv[7], sc.deriv[4], sc.deriv[5]]
        T = lambda a: torch.tensor(np.stack(a), dtype=torch.float64, device="cuda").contiguous()
        return T(st), T([sc.b, sc.deriv[6], sc.deriv[7]])
    sc, osc = S.adjoint_case(n), S.adjoint_case(n, hump_seed=1)
    gidx = S.gauges(n, n)
    solver = hw.Solver.from_scenario(sc, hw.make_params())
    state, static = eq(sc)
    dts = []
    for _ in range(nsteps):
        dt = solver.cfl_dt()
        dts.append(dt)
        solver.rk3_step(dt)
    osolver = hw.Solver.from_scenario(osc, hw.make_params())
    ostate, ostatic = eq(osc)
    A.load_problem(osolver, ostate, ostatic)
    _, gv = A.hw_gauge_loss(osolver.h, dts, gidx, np.zeros(nsteps * len(gidx)))
    obs = gv.ravel()
    osolver.close()
    A.load_problem(solver, state, static)
    A.hw_gauge_loss(solver.h, dts[:4], gidx, obs[:4 * len(gidx)])  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss_f, _ = A.hw_gauge_loss(solver.h, dts, gidx, obs)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    gs = torch.empty_like(state)
    gb = torch.empty_like(static)
    out = {"grid": [n, n], "steps": nsteps, "gauges": int(len(gidx)), "forward_s": t_fwd,
           "loss_forward_only": loss_f, "unit": "adjoint run time / forward loss time"}
    step_f = t_fwd / nsteps
    for name, snaps in (("tape", A.HW_ADJ_TAPE), ("checkpointed", snapshots)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss_a, nf = A.hw_adjoint_run(solver.h, dts, gidx, obs, snaps, [gs[q] for q in range(9)],
                                      [gb[q] for q in range(3)])
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        out[name] = {"snapshots": "every stage of every step" if snaps < 0 else snaps, "loss": loss_a,
                     "adjoint_run_s": t_adj, "adjoint_run_over_forward": t_adj / t_fwd,
                     "forward_steps_in_adjoint_run": int(nf),
                     "reverse_step_over_forward_step": (t_adj - nf * step_f) / nsteps / step_f,
                     "grad_norm_state": float(gs.norm()), "grad_norm_static": float(gb.norm())}
    solver.close()
    return out


def decomposed_compare(steps, splits=((2, 2), (4, 2))):
    """The benchmark workload split into blocks on this GPU (hw_dd_*: halo exchange between the blocks on
    the device, alpha as the maximum over blocks, two steps per CUDA graph): point-updates/s per split next
    to the undecomposed solver, and whether the states agree bit for bit."""
    import torch
    import paper_2208_01260_gb300 as hw
    from paper_2208_01260_gb300 import scenarios as S
    sc = S.bumps2d(NX, NY, strip=0.01)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(obj):
        obj.advance(4)
        torch.cuda.synchronize()
        e0.record(stream)
        obj.advance(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    s = hw.Solver.from_scenario(sc, hw.make_params())
    ms_single = timed(s)
    ref = s.state()
    s.close()
    out = {"steps": steps, "ms_per_step_single": ms_single, "unit": UNIT,
           "value_single": NX * NY * STAGES / (ms_single * 1e-3), "splits": {}}
    for px, py in splits:
        d = hw.DecomposedSolver(sc, px, py)
        ms = timed(d)
        got = d.state()
        d.close()
        out["splits"]["%dx%d" % (px, py)] = {
            "ms_per_step": ms, "value": NX * NY * STAGES / (ms * 1e-3), "over_single": ms_single / ms,
            "bitwise_equal_to_single": all(np.array_equal(a, b) for a, b in zip(ref, got))}
    out["adjoint"] = decomposed_adjoint_compare()
    return out


def decomposed_adjoint_compare(n=512, nsteps=100, px=2, py=2):
    """The gauge-misfit gradient of the adjoint workload (512^2, 32 gauges) over 2 x 2 blocks against the
    undecomposed adjoint, both on whole-run tapes: run times and the largest gradient difference."""
    import torch
    import paper_2208_01260_gb300 as hw
    from paper_2208_01260_gb300 import adjoint as A
    from paper_2208_01260_gb300 import scenarios as S
    sc = S.adjoint_case(n)
    gidx = S.gauges(n, n)
    solver = hw.Solver.from_scenario(sc, hw.make_params())
    dts = [solver.cfl_dt()] * nsteps
    obs = np.full(nsteps * len(gidx), 1.0)
    gs = torch.empty(9, n, n, dtype=torch.float64, device="cuda")
    gb = torch.empty(3, n, n, dtype=torch.float64, device="cuda")
    A.hw_adjoint_run(solver.h, dts[:2], gidx, obs[:2 * len(gidx)], A.HW_ADJ_TAPE, list(gs), list(gb))  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss, _ = A.hw_adjoint_run(solver.h, dts, gidx, obs, A.HW_ADJ_TAPE, list(gs), list(gb))
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    solver.close()
    d = hw.DecomposedSolver(sc, px, py)
    ds, db = torch.empty_like(gs), torch.empty_like(gb)
    hw.hw_dd_adjoint_run(d.h, dts[:2], gidx, obs[:2 * len(gidx)], list(ds), list(db))  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss_dd = hw.hw_dd_adjoint_run(d.h, dts, gidx, obs, list(ds), list(db))
    torch.cuda.synchronize()
    t_dd = time.perf_counter() - t0
    d.close()
    scale = float(gs.abs().max())
    return {"grid": [n, n], "steps": nsteps, "blocks": [px, py], "adjoint_run_s_single": t_single,
            "adjoint_run_s_blocks": t_dd, "blocks_over_single": t_dd / t_single, "loss_equal": loss == loss_dd,
            "max_grad_diff_over_largest": max(float((ds - gs).abs().max()), float((db - gb).abs().max())) / scale}


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2208_01260_gb300 import scenarios as S
    sc = S.bumps2d(NX, NY, strip=0.01)
    g = oracle.make_grid(sc.nx, sc.ny, sc.x0, sc.x1, sc.y0, sc.y1, sc.bc_x, sc.bc_y)
    p = oracle.make_params()
    st, stat = oracle.to_state2d(sc.h, sc.hu, sc.hv, sc.b, sc.deriv)
    # a reference step is one RK stage of the full grid (a bounded sample of one RK3 step)
    dt = oracle.cfl_dt2d(g, p, st, stat)
    cur, base = st, None
    k = 0
    for _ in range(args.warmup):
        cur, base, _ = oracle.stage2d(g, p, k % 3 + 1, dt, cur, stat, base)
        k += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cur, base, _ = oracle.stage2d(g, p, k % 3 + 1, dt, cur, stat, base if k % 3 else None)
        k += 1
    el = time.perf_counter() - t0
    value = NX * NY * args.steps / el
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "step": "one RK stage of the full grid (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "each step = one SSP-RK3 stage over the full 2048x2048 grid"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--batched-steps", type=int, default=6, help="steps of the batched comparison (0 = skip)")
    ap.add_argument("--batched-instances", type=int, default=512,
                    help="instances of the batched comparison (512: the benchmark workload; fewer for a small "
                         "case to profile)")
    ap.add_argument("--adjoint-steps", type=int, default=400, help="steps of the adjoint cost measurement (0 = skip)")
    ap.add_argument("--fp32-steps", type=int, default=200, help="steps of the single-precision variant (0 = skip)")
    ap.add_argument("--decomp-steps", type=int, default=10, help="steps of the block-decomposition comparison (0 = skip)")
    ap.add_argument("--onedim-reps", type=int, default=5, help="timed runs of each 1D run (0 = skip)")
    ap.add_argument("--nx", type=int, default=2048, help="smaller grids for profiling captures only")
    ap.add_argument("--ny", type=int, default=2048)
    args = ap.parse_args()
    global NX, NY, STATE_BYTES
    NX, NY = args.nx, args.ny
    STATE_BYTES = 9 * NX * NY * 8
    UNITS_PER_LAUNCH.update(sweep_x=(NX + 1) * NY, sweep_y=NX * (NY + 1), node=NX * NY, alpha=NX * NY)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ws, rank, local = dist_setup("nccl")
    import paper_2208_01260_gb300 as hw
    from paper_2208_01260_gb300 import scenarios as S

    # the FP64 roofline's denominator, measured on this GPU before the timed regions
    global PEAK_FP64_TFLOPS, PEAK_FP64_OPS
    with ClockSampler(local) as pclk:
        best, median, peak_ms = hw.hw_measure_fp64_peak(20)
    PEAK_FP64_OPS = median
    PEAK_FP64_TFLOPS = 2.0 * median / 1e12
    fp64_peak = {"fma_per_s_median": median, "fma_per_s_best": best, "tflops": PEAK_FP64_TFLOPS,
                 "launch_ms": peak_ms, "clocks": pclk.summary(), "nominal_tflops": NOMINAL_FP64_TFLOPS,
                 "how": "hw_measure_fp64_peak: 8 independent fma chains per thread, 8 x 256 threads per SM on "
                        "every SM, 4096 iterations, median of 20 event-timed launches (fma = 2 flops)"}

    sc = S.bumps2d(NX, NY, strip=0.01)
    solver = hw.Solver.from_scenario(sc, hw.make_params())
    if (NX, NY) != (2048, 2048):
        args.no_cpu_baseline = True
    stream = torch.cuda.current_stream()

    # warm-up (CUDA graph of two steps)
    solver.advance(args.warmup, use_graph=True)
    torch.cuda.synchronize()

    # timed region 1: K steps from the captured graph (production path)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        solver.advance(args.steps, use_graph=True)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    ms = ev0.elapsed_time(ev1)
    value, sec, _ = job_rate(NX * NY * STAGES * args.steps, ms * 1e-3, ws)
    ms = sec * 1e3

    # timed region 2: the same K steps with every kernel bracketed by events (per-kernel roofline)
    hw.hw_set_profiling(solver.h, True)
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.advance(args.steps, use_graph=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_prof = e0.elapsed_time(e1)
    prof = hw.hw_get_profile(solver.h)
    hw.hw_set_profiling(solver.h, False)
    launches_per_step = sum(n for _, n in prof.values()) / args.steps

    sha = sources_sha()
    hbm, hbm_src = hbm_peak()
    kernels = {}
    for k in ("sweep_x", "sweep_y", "node", "alpha"):
        tot, n = prof[k]
        if n == 0:
            continue
        nl = n if k != "alpha" else prof["sweep_x"][1]  # alpha: its kernels once per stage
        avg_s = tot / nl * 1e-3
        units = UNITS_PER_LAUNCH[k]
        tf = ALGO[k]["flops"] * units / avg_s / 1e12
        tr = TRAFFIC.get(k)
        traffic = tr["bytes_per_unit"] * units if tr and tr["sha"] == sha else None
        fp = FP64_PIPE_OPS.get(k)
        pipe_ops = fp["ops_per_unit"] if fp and fp["sha"] == sha else None
        kernels[k] = {"ms_avg": avg_s * 1e3, "launches": n, "share": tot / ms_prof, "tflops": tf,
                      "frac": tf / PEAK_FP64_TFLOPS,
                      "algo_ops_frac": ALGO[k]["ops"] * units / avg_s / PEAK_FP64_OPS,
                      "fp64_pipe_frac": (pipe_ops * units / avg_s / PEAK_FP64_OPS) if pipe_ops else None,
                      "traffic_bytes": traffic,
                      "hbm_frac": (traffic / avg_s / 1e9 / hbm) if traffic else None}
    dom = max(kernels, key=lambda k: kernels[k]["share"])
    kd = kernels[dom]
    roofline = {"bound": "alu", "achieved": kd["tflops"], "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": kd["frac"], "traffic": kd["traffic_bytes"], "kernel": "k_" + dom,
                "peak_src": "measured",
                "peak_how": "FP64 fma throughput measured live on this GPU before the timed region "
                            "(hw_measure_fp64_peak, median of 20 launches; fma = 2 flops); see fp64_peak",
                "algo_ops_frac": kd["algo_ops_frac"], "fp64_pipe_frac": kd["fp64_pipe_frac"],
                "int_pipe_note": "part of the products run on the integer pipes (bit-identical binary64), so the "
                                 "algorithmic rate can exceed the FP64 pipe's share; fp64_pipe_frac is the pipe's own use",
                "hbm_peak_gbs": hbm, "hbm_peak_src": hbm_src,
                "sources_sha": sha}
    step_ops = sum(ALGO[k]["ops"] * UNITS_PER_LAUNCH[k] for k in ALGO) * STAGES
    step_flops = sum(ALGO[k]["flops"] * UNITS_PER_LAUNCH[k] for k in ALGO) * STAGES
    step_s = ms / args.steps * 1e-3
    roofline["whole_step"] = {"tflops": step_flops / step_s / 1e12,
                              "frac": step_flops / step_s / 1e12 / PEAK_FP64_TFLOPS,
                              "algo_ops_frac": step_ops / step_s / PEAK_FP64_OPS}
    # the HBM roofline of the whole step: the algorithmic bytes a fused stage must move (216 B per node
    # and stage) over the step time, against the measured copy bandwidth; next to it the bytes this design
    # actually moves per node and stage (interfaces go through HBM so that no FP64 work is recomputed),
    # from the ncu traffic of the three kernels when the sources match the capture
    tr_node = None
    if all(TRAFFIC[k]["sha"] == sha for k in ("sweep_x", "sweep_y", "node")):
        tr_node = (TRAFFIC["sweep_x"]["bytes_per_unit"] * UNITS_PER_LAUNCH["sweep_x"]
                   + TRAFFIC["sweep_y"]["bytes_per_unit"] * UNITS_PER_LAUNCH["sweep_y"]
                   + TRAFFIC["node"]["bytes_per_unit"] * UNITS_PER_LAUNCH["node"]) / (NX * NY) + 2 * 32.0
    roofline["hbm_frac_step"] = ALGO_BYTES_PER_NODE_STAGE * NX * NY * STAGES / step_s / 1e9 / hbm
    roofline["hbm_step"] = {"algorithmic_bytes_per_node_stage": ALGO_BYTES_PER_NODE_STAGE,
                            "algorithmic_gbs": ALGO_BYTES_PER_NODE_STAGE * NX * NY * STAGES / step_s / 1e9,
                            "measured_dram_bytes_per_node_stage": tr_node,
                            "measured_dram_gbs": (tr_node * NX * NY * STAGES / step_s / 1e9) if tr_node else None,
                            "note": "bound: FP64 pipe, not HBM; the interface planes go through HBM by design"}

    # e2e through the public API with pinned host buffers: each step uploads the state (physical
    # layout, 9 planes), advances one RK3 step and downloads the state.
    host_in = [torch.empty(NY, NX, dtype=torch.float64).pin_memory() for _ in range(9)]
    host_out = [torch.empty(NY, NX, dtype=torch.float64).pin_memory() for _ in range(9)]
    hin = [t.numpy() for t in host_in]
    hout = [t.numpy() for t in host_out]
    hw.hw_get_state(solver.h, hout, hw.HW_LAYOUT_PHYSICAL)
    for a, b in zip(hin, hout):
        a[...] = b
    ke = max(1, min(args.e2e_steps, args.steps))
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        hw.hw_set_state(solver.h, hin, hw.HW_LAYOUT_PHYSICAL)
        solver.advance(1, use_graph=False)
        hw.hw_get_state(solver.h, hout, hw.HW_LAYOUT_PHYSICAL)
    torch.cuda.synchronize()
    e2e_serial, _, _ = job_rate(NX * NY * STAGES * ke, time.perf_counter() - t0, ws)
    # the same jobs (state up, one step, state down) through the pipelines of pipeline.py: two solvers on
    # their own streams and host threads (JobPipeline, the figure), and one solver whose copies run on an
    # upload and a download stream during the neighbouring jobs' steps (StagedPipeline)
    from paper_2208_01260_gb300.pipeline import JobPipeline, StagedPipeline
    outs = [[torch.empty(NY, NX, dtype=torch.float64).pin_memory().numpy() for _ in range(9)] for _ in range(2)]
    kp = max(4, ke)

    def pipeline_runs(pipe):
        pipe.run([hin] * 2, outs)  # warm-up
        # three timed runs of kp jobs each; the median run is the figure
        runs = []
        for _ in range(3):
            barrier(ws)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pipe.run([hin] * kp, [outs[i % 2] for i in range(kp)])
            torch.cuda.synchronize()
            runs.append(job_rate(NX * NY * STAGES * kp, time.perf_counter() - t0, ws)[0])
        pipe.close()
        return runs
    runs = pipeline_runs(JobPipeline(sc, hw.make_params(), lanes=2))
    runs2 = pipeline_runs(StagedPipeline(sc, hw.make_params()))
    e2e_v = statistics.median(runs)
    e2e = {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": STATE_BYTES,
           "d2h_bytes_per_step": STATE_BYTES, "steps": kp, "runs": runs,
           "how": "independent jobs (the 9-plane state uploaded from pinned host memory, one RK3 step, the state "
                  "downloaded), two solvers on their own streams and host threads (pipeline.JobPipeline); "
                  "median of three timed runs of `steps` jobs",
           "staged": {"value": statistics.median(runs2), "runs": runs2, "steps": kp,
                      "how": "the same jobs through one solver whose uploads and downloads run on their own streams "
                             "through two device staging sets each way, while the neighbouring jobs step "
                             "(pipeline.StagedPipeline: half the device memory)"},
           "serial": {"value": e2e_serial, "steps": ke,
                      "how": "one solver: upload, step, download, one job after the other"}}

    solver.sync()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "stages_per_step": STAGES,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "inputs larger than L2 (state 302 MB + interface planes 806 MB per grid)",
                       "timed_path": "hw_advance with a captured CUDA graph (2 steps per graph)"},
            "roofline": roofline, "kernels": kernels, "ms_per_step_profiled": ms_prof / args.steps,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clk.summary(), "e2e": e2e, "fp64_peak": fp64_peak}
    # secondary measurements: a failure is reported in the line instead of losing the headline
    def extra(key, fn):
        try:
            line[key] = fn()
        except Exception as exc:  # noqa: BLE001
            line[key] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    # (only in single-GPU runs: a scaling run measures the headline alone)
    if ws > 1:
        args.batched_steps = args.adjoint_steps = args.fp32_steps = args.decomp_steps = args.onedim_reps = 0
    if args.batched_steps > 0 and (NX, NY) == (2048, 2048):
        solver.close()
        extra("batched", lambda: dict(batched_compare(args.batched_steps, n_inst=args.batched_instances),
                                      **({} if args.batched_instances == 512 else
                                         {"workload": "%d grids drawn as the benchmark's (sizes log-uniform in [64, 1024]; not config 4)"
                                                      % args.batched_instances})))
        # the regime the batched form is for: grids too small to fill the GPU one launch at a time
        extra("batched_small_grids", lambda: dict(batched_compare(args.batched_steps, n_inst=1024, fixed=(64, 64)),
                                                  workload="1024 grids of 64x64 (not config 4)"))
    if args.decomp_steps > 0 and (NX, NY) == (2048, 2048):
        extra("decomposed", lambda: decomposed_compare(args.decomp_steps))
    if args.adjoint_steps > 0 and (NX, NY) == (2048, 2048):
        extra("adjoint", lambda: adjoint_cost(nsteps=args.adjoint_steps))
    if args.fp32_steps > 0:
        extra("fp32", lambda: fp32_variant(args.fp32_steps))
    if args.onedim_reps > 0:
        extra("onedim", lambda: onedim(args.onedim_reps))
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        def cpu():
            rate, desc, threads, el = oracle_rate()
            out = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc, "seconds": el}
            if args.onedim_reps > 0:
                out["onedim"] = oracle_onedim()
            return out
        extra("cpu_baseline", cpu)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
