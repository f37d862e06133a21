#!/usr/bin/env python
"""Benchmark of the LES hot path: grid-point RK-step updates per second.

A step is one full time step of the method (viscosity, time step, five
Runge-Kutta stages of the residual, boundary conditions) on the jet workload
288 x 160 x 128 (5.9M points, the size of the paper's Mesh A), Re_D = 1e5,
Mach 1.4, CFL 0.5, Smagorinsky SGS, synthetic seeded initial state resident
in HBM.  The headline is the FP32-mixed form; the FP64 form is measured on
the same GPU and reported beside it with the mixed form's error against it.

Contract: rank 0 prints one JSON line.  ``--impl reference`` times the CPU
oracle (the only other implementation of the method) on the host cores.
Multi-GPU runs are independent replicas (the path does not exchange data on
one node here): value = all ranks' point-steps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpt·RK-steps/s FP32-mixed vs FP64 at stated error, %HBM peak; adjoint/fwd ratio"
UNIT = "Gpt*RK-steps/s"
WORKLOAD = (288, 160, 128)
WORKLOAD_NAME = "jet 288x160x128 (5.9M pts, Mesh-A size), Re_D 1e5, M_j 1.4, CFL 0.5, Smagorinsky"

# Algorithmic bytes per grid point of one launch of each kernel class (what
# the kernel must read and write at least once, halos assumed cached), as
# (FP64, mixed), mean over the five stages of a step.  stage_fused: state in
# (Q or stage buffer), Q^(0) for the update, metrics (10), mu/kappa (2) and
# the stage state out.  FP64: 176 (stage 1), 216 (stages 2-5).  Mixed, the
# scope table's count: FP64 Q^(0) (40) read by every stage, float stage
# states, metrics and mu/kappa: 108, 128 x 3, 148 -> 128.  prestep: Q^n +
# metrics in, mu/kappa out.
BYTES_PER_POINT = {
    "stage_fused": ((176 + 4 * 216) / 5, (108 + 3 * 128 + 148) / 5),
    "prestep": (40 + 80 + 16, 20 + 40 + 8),
}
# The mixed kernel's own floor: it holds Q^(0) as a float pair (hi, lo) and
# stages 2-4 read only hi (20 B) for their update; the first stage reads no
# Q^(0) and the last reads and writes both parts: 88, 108 x 3, 148 -> 112.
BYTES_PER_POINT_FLOOR_MIXED = (88 + 3 * 108 + 148) / 5


# Counters of k_stage_fused from ncu captures on the 96 x 160 x 128 jet
# (per grid point; traffic and instruction counts grow in proportion to the
# points): DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum), mean
# over the five stages of a step, and FP32 add + mul + 2 x FMA.  Each figure
# describes the kernel source it was taken on only: bench.py reports it
# while the hash of that source still matches.
NCU_SOURCES = {"stage_fused": ("paper_2301_00817_gb300/csrc/fused_kernel.cuh",
                               "paper_2301_00817_gb300/csrc/fused.cu",
                               "paper_2301_00817_gb300/csrc/fused_jet12.cu",
                               "paper_2301_00817_gb300/csrc/fused_jet28.cu",
                               "paper_2301_00817_gb300/csrc/lesjet_dev.cuh"),
               "flux64": ("paper_2301_00817_gb300/csrc/stage64_kernels.cuh",
                          "paper_2301_00817_gb300/csrc/lesjet_dev.cuh")}
NCU_COUNTS = {
    ("stage_fused", "bytes_per_point"):
        (110.3, "08df13b959e108751e505c1ef6bdf6dc91de424d158d5a12d9a13d3b84a7ca2a"),
    ("stage_fused", "fp32_flop_per_point"):
        (1030, "08df13b959e108751e505c1ef6bdf6dc91de424d158d5a12d9a13d3b84a7ca2a"),
    # smsp__inst_executed.sum x 32 per point, mean of the five stages
    ("stage_fused", "inst_per_point"):
        (1605, "08df13b959e108751e505c1ef6bdf6dc91de424d158d5a12d9a13d3b84a7ca2a"),
    # FP64 flop (dadd + 2 x dfma + dmul) per grid point of one residual's
    # flux group on the 96 x 160 x 128 jet: k_sensor 64 + k_flux 260 + 259
    # + 257
    ("flux64", "fp64_flop_per_point"):
        (840, "e63f4edca7b4abbcc9117f9e6a9c50273f8fd20840063d4a79cfc30f512a18f5"),
}
NCU_CAPTURE = {"stage_fused": "profiles/stage_fused_jet96x160x128.md",
               "flux64": "profiles/flux64_jet96x160x128.md"}


def fp64_peak_from_units(clock_mhz=2070.0):
    """FP64 peak derived from the unit counts: the device's SMs x 2 DFMA per
    cycle x 2 flop x the SM clock (GB300: 152 SMs, 2.07 GHz maximum)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 2 * 2 * clock_mhz * 1e6 / 1e12


def traffic_per_point(kernel, field="bytes_per_point"):
    import hashlib
    rec = NCU_COUNTS.get((kernel, field))
    if rec is None:
        return None
    h = hashlib.sha256()
    try:
        for f in NCU_SOURCES[kernel]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return rec[0] if h.hexdigest() == rec[1] else None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms; only the
    samples stamped inside the timed region (mark_begin .. mark_end) count."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        self.dev = device_index
        self.t0 = self.t1 = None

    def start(self):
        try:
            import torch
            uuid = "GPU-" + str(torch.cuda.get_device_properties(self.dev).uuid)
        except Exception:
            uuid = None
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # wait for the first sample so that the timed region is covered
        deadline = time.time() + 10.0
        while time.time() < deadline and os.path.getsize(self.path) == 0:
            time.sleep(0.05)

    def mark_begin(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text):
        import datetime
        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)  # let the sample after the timed region land
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append((self._stamp(parts[0]), float(parts[2]), float(parts[3]),
                             float(parts[4]),
                             {nm for nm, v in zip(names, parts[6:10]) if v.lower().startswith("active")}))
            except ValueError:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if r[0] is not None and self.t0 is not None and
                  self.t0 - 0.05 <= r[0] <= self.t1 + 0.1]
        window = "timed region"
        if not inside:
            inside, window = rows, "whole sampler run (no sample stamped inside the timed region)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside),
                "power_w_max": max(r[3] for r in inside), "samples": len(inside),
                "window": window, "reasons": sorted(set().union(*(r[4] for r in inside)))}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    """Largest value over the ranks (the slowest replica's time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, points: int, steps: int, ms: float) -> float:
    """Whole-job Gpt*RK-steps/s: every replica advances `points` for `steps`
    steps; `ms` is the max-over-ranks time of the timed region."""
    return world * points * steps / (ms / 1e3) / 1e9


def oracle_baseline(shape, steps: int, warmup: int, threads: int = 0, grid=WORKLOAD, Re=1.0e5):
    """CPU oracle on an axial slab of the workload (same grid spacing and
    flow), all host cores (or `threads`); returns (Gpt*steps/s, seconds per
    step, points, threads used)."""
    import numpy as np

    import oracle
    full = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    from paper_2301_00817_gb300 import synth
    x, r, th = synth.jet_lines(*grid)
    ns = shape
    xyz = np.empty((3,) + ns)
    xyz[0] = x[:ns[0], None, None]
    xyz[1] = r[None, :, None] * np.cos(th)[None, None, :]
    xyz[2] = r[None, :, None] * np.sin(th)[None, None, :]
    P = oracle.params(sgs_model=1, Re=Re)
    M = oracle.metrics(xyz, (0, 0, 1))
    Q = oracle.init_jet(P, xyz, seed=0)
    t = 0.0
    for _ in range(warmup):
        Q, d = oracle.rk_step(P, Q, M, xyz, t)
        t += d
    t0 = time.perf_counter()
    for _ in range(steps):
        Q, d = oracle.rk_step(P, Q, M, xyz, t)
        t += d
    el = time.perf_counter() - t0
    npts = ns[0] * ns[1] * ns[2]
    used = oracle.num_threads()
    oracle.set_num_threads(full)
    return npts * steps / el / 1e9, el / steps, npts, used


def workload_config(world):
    """The config object of both arms' JSON lines (the same workload)."""
    N = WORKLOAD[0] * WORKLOAD[1] * WORKLOAD[2]
    return {"workload": WORKLOAD_NAME, "points": N, "global_batch": world, "seq_len": 0,
            "parallelism": f"replicas x{world}",
            "l2": "state and metrics (~0.9 GB) exceed the 129 MB L2; no flush needed"}


def run_reference(args, world, rank):
    """The oracle (plain FP64 C, OpenMP over nodes) on the host cores, on the
    whole workload: every timed step is one full RK step of all 5.9M points
    (about 2.3 s on 16 Grace cores)."""
    if rank != 0:
        return 0
    val, sec, npts, cores = oracle_baseline(WORKLOAD, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(1),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full RK steps of the whole workload "
                                   f"({npts} points), all host threads"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_steps(lj, torch, ctx, Q, steps, stream):
    """Device time of `steps` full steps through les_run_n_steps."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    diag = ctx.les_run_n_steps(steps, Q, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), diag


ADJ_WORKLOAD = (192, 96, 128)
ADJ_STEPS, ADJ_CKPT = 50, 10


def adjoint_leg(lj, torch, local):
    """Adjoint/forward cost on the jet 192 x 96 x 128 window: 50 FP64 steps,
    checkpoint every 10, 16 seeded forcing amplitudes, functional on the
    eta-surface nearest r = 5 D, no SGS model, fixed time step (the CFL step
    of the initial state).  Forward = les_run_n_steps over the window;
    adjoint = les_adjoint_window (forward sweep with checkpoints, segment
    recompute, reverse sweep)."""
    import numpy as np
    shape = ADJ_WORKLOAD
    xyz = torch.from_numpy(lj.synth.jet_grid(*shape)).cuda()
    amps = tuple(lj.synth.forcing_amplitudes(0))
    ctx = lj.Context(lj.make_params(precision=lj.PREC_FP64, sgs_model=lj.SGS_NONE, amp=amps),
                     shape, f"cuda:{local}")
    ctx.les_set_grid(xyz)
    Q0 = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
    ctx.les_init_jet(xyz, 0, 1e-3, Q0)
    dt = ctx.les_time_step(Q0)
    ctx.les_set_params(lj.make_params(precision=lj.PREC_FP64, sgs_model=lj.SGS_NONE, amp=amps,
                                      dt_mode=lj.DT_FIXED, dt_fixed=dt))
    j5 = int(np.argmin(np.abs(lj.synth.jet_radial(shape[1]) - 5.0)))
    aw = ctx.adjoint_workspace(ADJ_STEPS, ADJ_CKPT)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()

    def fwd():
        Q = Q0.clone()
        ctx.les_set_time(0.0)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.les_run_n_steps(ADJ_STEPS, Q)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def adj():
        torch.cuda.synchronize()
        e0.record(stream)
        J, g = ctx.les_adjoint_window(Q0, 0.0, ADJ_STEPS, ADJ_CKPT, j5, aw)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), J, g

    fwd(), adj()  # warm-up
    t_f = min(fwd() for _ in range(3))
    runs = [adj() for _ in range(3)]
    t_a, J, g = min(runs, key=lambda r: r[0])
    gnorm = float(np.linalg.norm(g))
    ws = aw.numel()
    # the same window with every stage state kept by the forward sweep (one
    # segment, no recompute): the memory-for-time end of the trade
    del aw
    aw = ctx.adjoint_workspace(ADJ_STEPS, ADJ_STEPS)
    ws_all = aw.numel()
    K = ADJ_STEPS

    def adj_all():
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.les_adjoint_window(Q0, 0.0, ADJ_STEPS, K, j5, aw)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    adj_all()
    t_all = min(adj_all() for _ in range(3))
    del aw
    # the same functional accumulated along an FP32-mixed forward run
    cm = lj.Context(lj.make_params(precision=lj.PREC_MIXED, sgs_model=lj.SGS_NONE, amp=amps,
                                   dt_mode=lj.DT_FIXED, dt_fixed=dt), shape, f"cuda:{local}")
    cm.les_set_grid(xyz)
    Qm = Q0.clone()
    cm.les_set_time(0.0)
    J_mixed = 0.0
    for _ in range(ADJ_STEPS):
        cm.les_run_n_steps(1, Qm)
        J_mixed += cm.les_surface_functional(Qm, j5, dt)
    del cm, Qm
    return {"workload": f"jet {shape[0]}x{shape[1]}x{shape[2]}, FP64, SGS none, "
                        f"{ADJ_STEPS}-step window, checkpoint every {ADJ_CKPT}",
            "functional": "sum_n dt sum_(i,k) (p - 1/gamma)^2 dA on the eta surface nearest r = 5",
            "dt": dt, "j_surface": j5, "forward_ms": t_f, "adjoint_window_ms": t_a,
            "ratio": t_a / t_f,
            "step_ratio": (t_a - t_f) / t_f,
            "ratio_note": "ratio: whole window (forward sweep with checkpoints + segment "
                          "recompute + reverse) over the forward run; step_ratio: the part "
                          "beyond the forward sweep, per step, over one forward step",
            "J": J, "grad_norm": gnorm, "workspace_gb": ws / 1e9,
            "J_mixed_forward": J_mixed, "J_mixed_rel_diff": abs(J_mixed - J) / abs(J),
            "store_all": {"adjoint_window_ms": t_all, "ratio": t_all / t_f,
                          "step_ratio": (t_all - t_f) / t_f,
                          "workspace_gb": ws_all / 1e9}}


LARGE_WORKLOAD = (2000, 500, 1024)
LARGE_SUBGRID = (1000, 250, 512)
LARGE_STEPS = 20


def _free_device_bytes(torch):
    import gc
    gc.collect()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def large_leg(lj, torch, local, hbm_peak, warmup):
    """The compact FP32-mixed form on the 2000 x 500 x 1024 jet (1.02e9
    points): 20 timed steps, the fused stage kernel's HBM fraction, device
    memory; and its error against FP64 after 20 steps on the 1/8-size
    1000 x 250 x 512 grid."""
    shape = LARGE_WORKLOAD
    N = shape[0] * shape[1] * shape[2]
    need = N * (40 + 129 + 24) + (4 << 30)
    free = _free_device_bytes(torch)
    if free < need:
        return {"skipped": f"needs {need / 1e9:.0f} GB free device memory, {free / 1e9:.0f} GB free"}
    stream = torch.cuda.current_stream()
    ctx = lj.Context(lj.make_params(sgs_model=lj.SGS_SMAGORINSKY,
                                    precision=lj.PREC_MIXED_COMPACT), shape, f"cuda:{local}")
    xyz = lj.synth.jet_grid_torch(*shape, f"cuda:{local}")
    ctx.les_set_grid(xyz)
    Q = torch.empty((5,) + shape, dtype=torch.float64, device=f"cuda:{local}")
    ctx.les_init_jet(xyz, 0, 1e-3, Q)
    del xyz
    torch.cuda.empty_cache()
    ctx.les_run_n_steps(warmup, Q)
    used = torch.cuda.memory_allocated()
    ctx.les_profile(True)
    ms, diag = time_steps(lj, torch, ctx, Q, LARGE_STEPS, stream)
    prof = ctx.les_profile_read()
    ctx.les_profile(False)
    ms_f, n_f = prof.get("stage_fused", (0.0, 0))
    bpp = BYTES_PER_POINT["stage_fused"][1]
    achieved = bpp * N / (ms_f / n_f / 1e3) / 1e9 if n_f else None
    out = {"workload": f"jet {shape[0]}x{shape[1]}x{shape[2]} ({N / 1e9:.2f}e9 points), "
                       "compact FP32-mixed (no FP64 metric copy), Smagorinsky",
           "value": N * LARGE_STEPS / (ms / 1e3) / 1e9, "unit": UNIT,
           "ms_per_step": ms / LARGE_STEPS, "status": diag.status,
           "device_gb_allocated": used / 1e9, "workspace_bytes_per_point": ctx.workspace.numel() / N,
           "stage_fused_hbm_frac": achieved / hbm_peak if achieved else None}
    del ctx, Q
    # error against FP64 on the 1/8-size grid
    sub = LARGE_SUBGRID
    xyz = lj.synth.jet_grid_torch(*sub, f"cuda:{local}")
    res = {}
    for prec in (lj.PREC_FP64, lj.PREC_MIXED_COMPACT):
        c = lj.Context(lj.make_params(sgs_model=lj.SGS_SMAGORINSKY, precision=prec), sub,
                       f"cuda:{local}")
        c.les_set_grid(xyz)
        Qs = torch.empty((5,) + sub, dtype=torch.float64, device=f"cuda:{local}")
        c.les_init_jet(xyz, 0, 1e-3, Qs)
        c.les_run_n_steps(LARGE_STEPS, Qs)
        res[prec] = Qs
        del c
    a, b = res[lj.PREC_MIXED_COMPACT], res[lj.PREC_FP64]
    out["error_vs_fp64_subgrid"] = {
        f"rel_l2_{nm}": float(torch.linalg.vector_norm(a[c] - b[c]) / torch.linalg.vector_norm(b[c]))
        for c, nm in ((0, "rho"), (1, "rho_u"), (4, "rho_E"))}
    out["error_vs_fp64_subgrid"]["grid"] = f"{sub[0]}x{sub[1]}x{sub[2]}, {LARGE_STEPS} steps"
    del res, a, b, xyz
    torch.cuda.empty_cache()
    return out


def extensions_leg(lj, torch, local, xyz, shape, base_ms, steps=10, warmup=2):
    """Cost of the options beyond the configured workload, on the same grid:
    the dynamic SGS model (FP64 and mixed), local time steps and the
    characteristic entrance (mixed), and the conservative metric setup."""
    stream = torch.cuda.current_stream()
    out = {"steps": steps}
    cases = (("fp64_dynamic", dict(precision=lj.PREC_FP64, sgs_model=lj.SGS_DYNAMIC)),
             ("mixed_local_dt", dict(precision=lj.PREC_MIXED, sgs_model=lj.SGS_SMAGORINSKY,
                                     dt_mode=lj.DT_LOCAL)),
             ("mixed_char_bc", dict(precision=lj.PREC_MIXED, sgs_model=lj.SGS_SMAGORINSKY,
                                    bc=lj.BC_JET_CHAR)),
             ("mixed_dynamic", dict(precision=lj.PREC_MIXED, sgs_model=lj.SGS_DYNAMIC)))
    for name, kw in cases:
        ctx = lj.Context(lj.make_params(**kw), shape, f"cuda:{local}")
        ctx.les_set_grid(xyz)
        Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
        ctx.les_init_jet(xyz, 0, 1e-3, Q)
        ctx.les_run_n_steps(warmup, Q)
        ctx.les_profile(True)
        ms, diag = time_steps(lj, torch, ctx, Q, steps, stream)
        prof = ctx.les_profile_read()
        ctx.les_profile(False)
        rec = {"ms_per_step": ms / steps, "status": diag.status,
               "kernel_ms_per_step": {k: v[0] / steps for k, v in prof.items() if v[1]}}
        ref = base_ms["fp64" if kw["precision"] == lj.PREC_FP64 else "mixed"]
        rec["vs_configured_step"] = rec["ms_per_step"] / ref
        if name in ("fp64_dynamic", "mixed_dynamic"):
            co = ctx.les_dynamic_coefficients(Q)
            rec["coefficients"] = {k: co[k] for k in ("Cd", "CI", "Prt")}
        out[name] = rec
        del ctx, Q
        torch.cuda.empty_cache()
    setup = {}
    for name, form in (("cross", lj.METRIC_CROSS), ("conservative", lj.METRIC_CONSERVATIVE)):
        ctx = lj.Context(lj.make_params(precision=lj.PREC_MIXED, metric_form=form), shape,
                         f"cuda:{local}")
        ctx.les_set_grid(xyz)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.les_set_grid(xyz)
        e1.record(stream)
        torch.cuda.synchronize()
        setup[name] = e0.elapsed_time(e1)
        del ctx
    out["set_grid_ms"] = setup
    return out


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2301_00817_gb300 as lj
    from paper_2301_00817_gb300 import _build

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    lj.load_library()
    shape = WORKLOAD
    N = shape[0] * shape[1] * shape[2]
    xyz = torch.from_numpy(lj.synth.jet_grid(*shape)).cuda()
    stream = torch.cuda.current_stream()
    hbm_peak, peak_src = load_peaks()
    fma_peaks = {"fp64": lj.measure_fma_peak(lj.PREC_FP64),
                 "fp32": lj.measure_fma_peak(lj.PREC_MIXED)}

    results = {}
    for name, prec in (("mixed", lj.PREC_MIXED), ("fp64", lj.PREC_FP64)):
        params = lj.make_params(sgs_model=lj.SGS_SMAGORINSKY, precision=prec)
        ctx = lj.Context(params, shape, f"cuda:{local}")
        ctx.les_set_grid(xyz)
        Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
        ctx.les_init_jet(xyz, 0, 1e-3, Q)
        ctx.les_run_n_steps(args.warmup, Q)
        ctx.les_profile(True)
        launches0 = ctx.les_launch_count()
        barrier(world)
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if name == "mixed" else None
        if sampler:
            sampler.start()
            sampler.mark_begin()
        ms, diag = time_steps(lj, torch, ctx, Q, args.steps, stream)
        if sampler:
            sampler.mark_end()
        clocks = sampler.stop() if sampler else None
        barrier(world)
        prof = ctx.les_profile_read()
        ctx.les_profile(False)
        launches = ctx.les_launch_count() - launches0
        ms = max_over_ranks(world, ms)
        results[name] = dict(ms=ms, diag=diag, prof=prof, launches=launches, clocks=clocks,
                             ctx=ctx, Q=Q)

    # e2e: the same step through the C ABI on a pinned host state
    ctx = results["mixed"]["ctx"]
    Qh = results["mixed"]["Q"].cpu().pin_memory()
    Qstage = torch.empty_like(results["mixed"]["Q"])
    ctx.les_run_host(1, Qh, Qstage)  # warm the copy path
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.les_run_host(1, Qh, Qstage)
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)

    # error of the mixed form against FP64 (same seed, 100 steps)
    err = None
    if not args.no_accuracy:
        outs = {}
        for name in ("fp64", "mixed"):
            c = results[name]["ctx"]
            Qa = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
            c.les_init_jet(xyz, 0, 1e-3, Qa)
            c.les_set_time(0.0)
            c.les_run_n_steps(args.accuracy_steps, Qa)
            outs[name] = Qa
        a, b = outs["mixed"], outs["fp64"]
        err = {f"rel_l2_{nm}": float(torch.linalg.vector_norm(a[c] - b[c]) /
                                     torch.linalg.vector_norm(b[c]))
               for c, nm in ((0, "rho"), (1, "rho_u"), (4, "rho_E"))}
        err["steps"] = args.accuracy_steps

    ext = None
    if not args.no_extensions and world == 1:
        base = {k: results[k]["ms"] / args.steps for k in ("mixed", "fp64")}
        ext = extensions_leg(lj, torch, local, xyz, shape, base)
    adj = None
    if not args.no_adjoint:
        adj = adjoint_leg(lj, torch, local)
    large = None
    if world > 1:
        large = {"skipped": "run at n_gpus = 1 only"}
    elif not args.no_large:
        for name in ("mixed", "fp64"):
            results[name].pop("ctx", None)
            results[name].pop("Q", None)
        del ctx, Qh, Qstage
        large = large_leg(lj, torch, local, hbm_peak, args.warmup)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, sec, npts, cores = oracle_baseline(WORKLOAD, 1, 0)
        slab = (24, WORKLOAD[1], WORKLOAD[2])
        v1, s1, n1, _ = oracle_baseline(slab, 1, 0, threads=1)
        cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
               "seconds": sec,
               "sample": f"1 full RK step of the whole workload ({npts} points), "
                         "all host threads",
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "seconds": s1,
                                 "sample": f"1 full RK step of the axial slab {slab} "
                                           f"({n1} points), one thread"}}

    def roofline(res, prec_idx):
        prof = res["prof"]
        top = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
        ms_tot, n_launch = prof[top]
        per_launch_s = ms_tot / n_launch / 1e3
        bpp = BYTES_PER_POINT.get(top, (None, None))[prec_idx]
        if bpp is None:
            return {"kernel": top, "bound": "hbm", "achieved": None, "peak": hbm_peak,
                    "unit": "GB/s", "frac": None, "traffic": None}
        achieved = bpp * N / per_launch_s / 1e9
        share = ms_tot / sum(v[0] for v in prof.values())
        tpp = traffic_per_point(top) if prec_idx == 1 else None
        out = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
               "unit": "GB/s", "frac": achieved / hbm_peak,
               "traffic": tpp * N if tpp is not None else None,
               "traffic_source": NCU_CAPTURE.get(top) if tpp is not None else None,
               "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, burst copy)",
               "bytes_per_point": bpp, "avg_launch_us": per_launch_s * 1e6,
               "share_of_step": share}
        if prec_idx == 1 and top == "stage_fused":
            fl = BYTES_PER_POINT_FLOOR_MIXED
            out["bytes_per_point_floor"] = fl
            out["frac_at_floor"] = fl * N / per_launch_s / 1e9 / hbm_peak
            out["floor_note"] = ("this kernel's own minimum: Q^(0) held as a float pair, stages "
                                 "2-4 read only its hi part")
        return out

    def roofline_fp64_alu(res):
        ms_tot, n_group = res["prof"].get("flux", (0.0, 0))
        fpp = traffic_per_point("flux64", "fp64_flop_per_point")
        if not n_group or fpp is None:
            return None
        per_group_s = ms_tot / n_group / 1e3
        achieved = fpp * N / per_group_s / 1e12
        peak = fma_peaks["fp64"]
        return {"kernel": "flux group (k_sensor + 3 x k_flux)", "bound": "alu", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": "measured FP64 FMA chains (les_measure_fma_peak); derived from unit "
                               f"counts: {fp64_peak_from_units():.3f}",
                "flop_per_point": fpp, "flop_source": NCU_CAPTURE["flux64"],
                "avg_group_us": per_group_s * 1e6}

    def roofline_fp32_alu(res):
        ms_tot, n_launch = res["prof"].get("stage_fused", (0.0, 0))
        fpp = traffic_per_point("stage_fused", "fp32_flop_per_point")
        if not n_launch or fpp is None:
            return None
        achieved = fpp * N / (ms_tot / n_launch / 1e3) / 1e12
        return {"kernel": "stage_fused", "bound": "alu", "achieved": achieved,
                "peak": fma_peaks["fp32"], "unit": "TFLOP/s", "frac": achieved / fma_peaks["fp32"],
                "peak_source": "measured FP32 FMA chains (les_measure_fma_peak)",
                "flop_per_point": fpp}

    def roofline_issue(res):
        # instruction issue: every SM issues at most one warp-instruction per
        # scheduler per clock (152 SMs x 4 schedulers on GB300), at the SM
        # clock sampled during the timed region
        ms_tot, n_launch = res["prof"].get("stage_fused", (0.0, 0))
        ipp = traffic_per_point("stage_fused", "inst_per_point")
        clk = (res.get("clocks") or {}).get("sm_mhz")
        if not n_launch or ipp is None or not clk:
            return None
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        peak = sms * 4 * clk * 1e6 / 1e9  # G warp-instructions/s
        achieved = ipp / 32.0 * N / (ms_tot / n_launch / 1e3) / 1e9
        return {"kernel": "stage_fused", "bound": "issue", "achieved": achieved, "peak": peak,
                "unit": "G warp-instructions/s", "frac": achieved / peak,
                "peak_source": f"{sms} SMs x 4 schedulers x {clk:.0f} MHz (sampled SM clock)",
                "inst_per_point": ipp}

    mixed, fp64 = results["mixed"], results["fp64"]
    ms_step = mixed["ms"] / args.steps
    value = aggregate_rate(world, N, args.steps, mixed["ms"])
    fp64_value = aggregate_rate(world, N, args.steps, fp64["ms"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": workload_config(world),
        "precision": "FP32 arithmetic (fluxes, dissipation, SGS); metrics built in FP64 and stored "
                     "FP32; Q^(0) as a compensated float pair (FP64-accurate RK accumulation)",
        "roofline": roofline(mixed, 1),
        "roofline_alu": roofline_fp32_alu(mixed),
        "roofline_issue": roofline_issue(mixed),
        "fma_peaks_tflops": fma_peaks,
        "cpu_baseline": cpu,
        "e2e": {"value": world * N * args.steps / e2e_s / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": 5 * N * 8, "d2h_bytes_per_step": 5 * N * 8,
                "api": "les_run_host (pinned host state in and out every step)"},
        "gpu_launches": mixed["launches"],
        "clocks": mixed["clocks"],
        "fp64": {"value": fp64_value, "ms_per_step": fp64["ms"] / args.steps, "dtype": "f64",
                 "roofline_alu": roofline_fp64_alu(fp64),
                 "gpu_launches": fp64["launches"]},
        "mixed_error_vs_fp64": err,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in mixed["prof"].items() if v[1]},
        "kernel_ms_per_step_fp64": {k: v[0] / args.steps for k, v in fp64["prof"].items() if v[1]},
        "extensions": ext,
        # the backward pass (segment recompute + reverse) over the forward
        # pass, per step; the whole window including the forward sweep is
        # adjoint_window_ratio
        "adjoint_fwd_ratio": adj["step_ratio"] if adj else None,
        "adjoint_window_ratio": adj["ratio"] if adj else None,
        "adjoint": adj,
        "large": large,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_profile_case(which: str):
    """Small case for ncu captures: 96 x 160 x 128 jet (1.97M points, state
    and metrics above the 129 MB L2), two full steps, one precision (the
    dynamic cases: FP64 or FP32-mixed with the dynamic SGS model); or the
    adjoint window on 96 x 96 x 128 (10 steps, checkpoint every 5)."""
    import numpy as np
    import torch

    import paper_2301_00817_gb300 as lj
    from paper_2301_00817_gb300 import _build
    _build.build()
    if which == "adjoint":
        shape = (96, 96, 128)
        amps = tuple(lj.synth.forcing_amplitudes(0))
        kw = dict(precision=lj.PREC_FP64, sgs_model=lj.SGS_NONE, amp=amps)
        ctx = lj.Context(lj.make_params(**kw), shape)
        xyz = torch.from_numpy(lj.synth.jet_grid(*shape)).cuda()
        ctx.les_set_grid(xyz)
        Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
        ctx.les_init_jet(xyz, 0, 1e-3, Q)
        dt = ctx.les_time_step(Q)
        ctx.les_set_params(lj.make_params(dt_mode=lj.DT_FIXED, dt_fixed=dt, **kw))
        j5 = int(np.argmin(np.abs(lj.synth.jet_radial(shape[1]) - 5.0)))
        aw = ctx.adjoint_workspace(10, 5)
        J, g = ctx.les_adjoint_window(Q, 0.0, 10, 5, j5, aw)
        print(f"profile case adjoint: J={J:.6e} |grad|={float(np.linalg.norm(g)):.3e} "
              f"launches={ctx.les_launch_count()}")
        return 0
    if which == "c3":
        # 576 x 320 x 256 (47M points), Re_D = 1e6: both forms, 5 timed steps
        # each after 2 warm-up steps, and one oracle step on the host cores
        shape = (576, 320, 256)
        N = shape[0] * shape[1] * shape[2]
        xyz = lj.synth.jet_grid_torch(*shape, "cuda")
        out = {"workload": "jet 576x320x256 (47.2M points), Re_D 1e6, Smagorinsky",
               "points": N}
        for name, prec in (("mixed", lj.PREC_MIXED), ("fp64", lj.PREC_FP64)):
            ctx = lj.Context(lj.make_params(Re=1.0e6, sgs_model=lj.SGS_SMAGORINSKY,
                                            precision=prec), shape)
            ctx.les_set_grid(xyz)
            Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
            ctx.les_init_jet(xyz, 0, 1e-3, Q)
            ctx.les_run_n_steps(2, Q)
            ctx.les_profile(True)
            ms, diag = time_steps(lj, torch, ctx, Q, 5, torch.cuda.current_stream())
            prof = ctx.les_profile_read()
            ctx.les_profile(False)
            rec = {"ms_per_step": ms / 5, "gpt_steps_per_s": N * 5 / (ms / 1e3) / 1e9,
                   "status": diag.status,
                   "kernel_ms_per_step": {k: v[0] / 5 for k, v in prof.items() if v[1]}}
            if name == "mixed":
                st = prof["stage_fused"]
                per_launch_s = st[0] / st[1] / 1e3
                rec["stage_fused_avg_launch_us"] = per_launch_s * 1e6
                rec["stage_fused_algorithmic_gbs"] = (BYTES_PER_POINT["stage_fused"][1] * N /
                                                      per_launch_s / 1e9)
            out[name] = rec
            del ctx, Q
            torch.cuda.empty_cache()
        del xyz
        val, sec, npts, cores = oracle_baseline(shape, 1, 0, grid=shape, Re=1.0e6)
        out["oracle_one_step"] = {"seconds": sec, "cores": cores, "gpt_steps_per_s": val}
        print(json.dumps(out))
        return 0
    prec = lj.PREC_MIXED if which in ("mixed", "dynamic_mixed") else lj.PREC_FP64
    sgs = lj.SGS_DYNAMIC if which in ("dynamic", "dynamic_mixed") else lj.SGS_SMAGORINSKY
    shape = (96, 160, 128)
    ctx = lj.Context(lj.make_params(sgs_model=sgs, precision=prec), shape)
    xyz = torch.from_numpy(lj.synth.jet_grid(*shape)).cuda()
    ctx.les_set_grid(xyz)
    Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
    ctx.les_init_jet(xyz, 0, 1e-3, Q)
    d = ctx.les_run_n_steps(2, Q)
    print(f"profile case {which}: t={d.t:.6e} dt={d.dt:.6e} launches={ctx.les_launch_count()}")
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--accuracy-steps", type=int, default=100)
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-extensions", action="store_true",
                    help="skip the dynamic-SGS / local-step / entrance / metric-form timings")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 1.02e9-point compact mixed leg")
    ap.add_argument("--profile-case", choices=("fp64", "mixed", "adjoint", "dynamic", "dynamic_mixed",
                                               "c3"),
                    default=None,
                    help="run the small ncu case (two steps) and exit")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args.profile_case)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
