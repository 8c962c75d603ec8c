#!/usr/bin/env python
"""Throughput of the GRMHD step on GB300: Mzone-updates/s per SSP-RK3 step.

Workload (default): the 256^3 periodic special-relativistic MHD box of
``inputs.sweep_box`` (rho in [0.5,1.5], log-uniform p in [0.1,1], |v| <= 0.6,
plasma beta ~1-100, Gamma = 4/3, CFL 0.4), FP64 throughout.  A step is one
whole SSP-RK3 step: three stages of ghost fill, c2p, MP5+HLL faces, UCT EMFs
and the update, with the CFL dt reduced on the device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision 64|32]
                  [--size 256] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (the
only other implementation of this method) on a bounded sample of the same
workload on this host's cores.  Under torchrun every rank runs an
independent replica (the step has no data exchange on one GPU per run).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mzone-updates/s per RK3 step"
UNIT = "Mzone/s"

# Algorithmic bytes per unit of each kernel class (FP64 values are 8 B; the
# FP32 path stores 4 B values except Z, which stays FP64).  Counts: every
# array element a kernel must read or write once (halo re-reads excluded).
#   c2p     per cell: read D,S,tau (5) + 3 face B + Z; write 8 primitives + Z
#   faces   per face: read 7 primitives + normal B; write 5 fluxes, a+, a-,
#           4 face velocities
#   emf     per edge: read 4 face velocities, 2 face B, 4 speeds; write E
#   update  per cell: read 15 fluxes, 3 EMFs, U (8), U0 (8); write U (8)
KMODEL = {
    "c2p": dict(vals=18, z=2),
    "faces_x": dict(vals=19), "faces_y": dict(vals=19), "faces_z": dict(vals=19),
    "emf_x": dict(vals=11), "emf_y": dict(vals=11), "emf_z": dict(vals=11),
    "update": dict(vals=42),
}


# The method's own FP64 operations per unit (the roofline numerator): read
# from oracle/op_counts.json, which the oracle's operation-counting build
# writes (oracle/count_ops.py: one step of this workload at 256^3 after the
# warm-up steps; +, -, *, / and sqrt each one operation, every distinct
# operation once per unit).  Read as data; nothing of the oracle runs here.
OP_COUNTS_PATH = os.path.join(ROOT, "oracle", "op_counts.json")


def load_op_counts(path=None):
    with open(path or OP_COUNTS_PATH) as f:
        return json.load(f)


def algorithmic_flops(counts, kernel, newton_iters):
    """The method's FP64 operations per unit of a kernel class: faces per
    face, EMFs per edge, update per cell (flux differences, CT curl, RK
    combination), c2p per cell at the inversion's Newton iterations (the
    oracle's count split into a part per cell and a part per iteration)."""
    f = counts["flops_per_unit"]
    if kernel.startswith("faces"):
        return f["faces"]
    if kernel.startswith("emf"):
        return f["emf"]
    if kernel == "update":
        return counts["update_per_cell"]
    if kernel == "c2p":
        return counts["c2p_per_cell_fixed"] + counts["c2p_per_newton_iteration"] * newton_iters
    return None


# The kernels' own FP64 floating-point operations per unit (context beside
# the algorithmic count): 2 x DFMA + DADD + DMUL thread instructions counted
# by ncu, including those inside divisions and square roots, on one launch at
# 128^3 of the same input recipe (sweep_box), divided by the units of that
# launch.  c2p depends on the Newton iteration count (2.74 per call there);
# faces_y/z run the code of faces_x with other strides.
FLOPS64 = {
    64: {"faces_x": 476.3, "faces_y": 476.3, "faces_z": 476.3,
         "emf_x": 236.4, "emf_y": 236.4, "emf_z": 236.4,
         "c2p": 359.5, "update": 79.0},
    # FP32-bulk path: only c2p computes in FP64 (previous-stage Z refined in
    # FP32, then 1.01 FP64 Newton iterations per call, the first with f'
    # from the FP32 refinement)
    32: {"c2p": 95.0},
}
# FP64-pipe thread instructions (DFMA + DADD + DMUL; ncu counts 64-bit
# integer adds, compares and masks with the DADDs, and the kernels keep
# those on 32-bit words) per unit from the same captures: each takes one
# lane slot of the FP64 pipe, so these over the pipe's nominal 2 lanes per
# SM and clock give the pipe-time view beside the flop roofline (DADD and
# DMUL are one flop for a full slot).
FP64_INSTR = {
    64: {"faces_x": 331.7, "faces_y": 331.7, "faces_z": 331.7, "emf_x": 167.8, "emf_y": 167.8, "emf_z": 167.8,
         "c2p": 251.3, "update": 53.0},
    32: {"c2p": 69.0},
}
# Nominal FP64 peak of the GB300 from its unit counts and clock: 152 SMs x 2
# DFMA lanes per SM and clock x 2 flop x 2.07 GHz (the 1.25 TFLOP/s figure);
# the roofline uses the rate measured by the library's FP64 FMA probe
# (measure_fp64_peak), this only if the probe cannot run.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def measure_fp64_peak(dev, repeats=3, iters=20000):
    """FP64 rate of the library's register-only FMA probe
    (echo_selftest_dfma, at the FP64 pipe's full issue rate), best of
    `repeats` launches timed with CUDA events after one untimed launch of the
    same length: (TFLOP/s, source)."""
    import torch
    from paper_1810_04597_gb300 import _lib
    try:
        blocks = _lib.echo_selftest_dfma_blocks()
        out = torch.empty(256 * blocks, dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream(dev)
        _lib.echo_selftest_dfma(iters, out, st.cuda_stream)   # warm-up as long as a timed launch
        best = 0.0
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            flops = _lib.echo_selftest_dfma(iters, out, st.cuda_stream)
            b.record(st)
            torch.cuda.synchronize()
            best = max(best, flops / (a.elapsed_time(b) * 1e-3) / 1e12)
        return best, "measured: FP64 FMA throughput probe (echo_selftest_dfma), best of %d launches" % repeats
    except Exception as exc:   # keep the bench line; say which peak it is
        return FP64_PEAK_TFLOPS, f"nominal (probe failed: {exc})"
# DRAM bytes per face of faces_x (dram__bytes_read.sum + dram__bytes_write.sum
# of the same 128^3 ncu launch: 337,239,040 B over 2,316,324 faces); scaled to a
# launch by the faces it processes.
TRAFFIC_PER_FACE64 = 337239040 / 2316324
# FP64 pipe activity in those captures
# (sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active).
FP64_PIPE_BUSY = {64: {"faces_x": 0.880, "faces_y": 0.880, "faces_z": 0.880, "emf_x": 0.874, "emf_y": 0.874,
                       "emf_z": 0.874, "c2p": 0.869, "update": 0.827},
                  32: {"c2p": 0.839}}
# The FP64 pipe's nominal lane rate (thread instructions per second): 152 SMs
# x 2 lanes per SM and clock x 2.07 GHz.  The FMA probe issues at 0.996 of
# it; FMAs that read three distinct 64-bit registers issue at 0.80-0.97.
FP64_PIPE_LANES_PER_S = 152 * 2 * 2.07e9


def fp64_mix_cap(flops_per_unit, fp64_instr_per_unit, peak_tflops):
    """Fraction of the FMA peak a kernel can reach with its own FP64
    instruction mix when the pipe issues on every lane slot: DADD and DMUL
    take a full slot for one flop, an FMA two."""
    return flops_per_unit / fp64_instr_per_unit * FP64_PIPE_LANES_PER_S / 1e12 / peak_tflops


def kernel_units(name, n):
    nx, ny, nz = n
    g = 3
    if name == "c2p" or name == "update":
        return nx * ny * nz
    if name == "faces_x":
        return (nx + 1) * (ny + 2 * g) * (nz + 2 * g)
    if name == "faces_y":
        return (nx + 2 * g) * (ny + 1) * (nz + 2 * g)
    if name == "faces_z":
        return (nx + 2 * g) * (ny + 2 * g) * (nz + 1)
    if name == "emf_x":
        return nx * (ny + 1) * (nz + 1)
    if name == "emf_y":
        return (nx + 1) * ny * (nz + 1)
    if name == "emf_z":
        return (nx + 1) * (ny + 1) * nz
    return 0


def kernel_bytes_per_unit(name, precision):
    m = KMODEL[name]
    size = 8 if precision == 64 else 4
    z = m.get("z", 0)
    return (m["vals"] - z) * size + z * 8


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=None):
        self.proc = None
        self.lines = []
        self.gpu_index = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r.split(",") for r in self.lines if r]
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if self.gpu_index is not None:
            sel = [r for r in rows if r[0] == str(self.gpu_index)]
            rows = sel or rows
        if rows:
            first = rows[0][0]
            rows = [r for r in rows if r[0] == first]

        def num(x):
            try:
                return float(x.split()[0])
            except Exception:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max([num(r[3]) for r in rows if num(r[3]) is not None], default=None)}


# ------------------------------------------------------------------ CPU oracle

def oracle_rate(prob, nsteps_hint, budget_s):
    """Time oracle SSP-RK3 steps of problem `prob` (FP64 C oracle, OpenMP
    over cells) for about budget_s seconds after one untimed step.
    Returns (zones_per_s, steps, seconds, threads)."""
    import oracle
    cfg = oracle.make_cfg(prob)
    st, Z = oracle.p2c(cfg, prob.prims, prob.bface)
    t0 = time.perf_counter()
    st, Z, _, _ = oracle.steps(cfg, st, Z, 1)
    t1 = time.perf_counter() - t0
    steps = max(1, min(nsteps_hint, int(budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.steps(cfg, st, Z, steps)
    dt = time.perf_counter() - t0
    return prob.ncells * steps / dt, steps, dt, oracle.get_threads()


def oracle_sample(prob, nsteps_hint, budget_s, w=48):
    """Time oracle SSP-RK3 steps on the workload's recipe at w^3 (a periodic
    sweep_box of the same seeded recipe) for about budget_s seconds.
    Returns (zones_per_s, zones, steps, seconds, threads, w)."""
    from paper_1810_04597_gb300 import inputs
    v, steps, dt, threads = oracle_rate(inputs.sweep_box(w), nsteps_hint, budget_s)
    return v, w ** 3, steps, dt, threads, w


def cpu_baseline_rows(budget_s):
    """The oracle on the host cores: the workload's recipe (sweep_box) on all
    cores at 80^3 and on one thread at 48^3, and the torus recipe
    (Fishbone-Moncrief, a = 0.9, beta 100, the 256x128x128 workload's
    recipe at 64x32x32) on all cores."""
    import oracle
    from paper_1810_04597_gb300 import inputs
    oracle.build()
    cores = oracle.get_threads()
    v, z, nsteps_c, secs, threads, w = oracle_sample(None, 50, budget_s, w=80)
    out = {"value": v / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"sweep_box recipe at {w}^3 (periodic), {nsteps_c} SSP-RK3 steps, "
                     f"{secs:.1f} s, FP64 C oracle with OpenMP over cells",
           "cpu": cpu_description()}
    oracle.set_threads(1)
    try:
        v1, s1, d1, t1 = oracle_rate(inputs.sweep_box(48), 20, budget_s / 3)
    finally:
        oracle.set_threads(cores)
    out["one_thread"] = {"value": v1 / 1e6, "unit": UNIT, "cores": t1,
                         "sample": f"sweep_box recipe at 48^3, {s1} steps, {d1:.1f} s, one thread"}
    tor = inputs.fm_torus((64, 32, 32), spin=0.9, beta=100.0)
    vt, st_, dtt, tt = oracle_rate(tor, 20, budget_s / 3)
    out["torus"] = {"value": vt / 1e6, "unit": UNIT, "cores": tt,
                    "sample": f"Fishbone-Moncrief torus (a = 0.9, beta 100, floors) at 64x32x32, {st_} steps, "
                              f"{dtt:.1f} s, all cores"}
    return out


def cpu_description():
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
        arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}
        ncpu = sum(1 for ln in txt.splitlines() if ln.startswith("processor"))
        for key in ("model name", "CPU part", "Hardware"):
            for ln in txt.splitlines():
                if ln.startswith(key):
                    v = ln.split(":", 1)[1].strip()
                    name = arm_parts.get(v, v) if key == "CPU part" else v
                    return f"{name} (CPU part {v})" if key == "CPU part" else name
        if ncpu:
            return f"{ncpu} processors"
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


# ------------------------------------------------------------------ distributed

def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, local):
    import torch
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        return dist
    return None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ arms

def workload_name(args):
    return (f"sweep_box {args.size}^3 periodic SRMHD, Gamma 4/3, CFL 0.4, "
            f"{'FP64' if args.precision == 64 else 'FP32 bulk'}")


def run_reference(args, world, rank):
    """The oracle (plain FP64 C, OpenMP over cells) as the reference arm."""
    if rank != 0:
        return None
    from paper_1810_04597_gb300 import inputs
    import oracle
    oracle.build()
    w = min(64, args.size)
    win = inputs.sweep_box(w)
    cfg = oracle.make_cfg(win)
    st, Z = oracle.p2c(cfg, win.prims, win.bface)
    st, Z, _, _ = oracle.steps(cfg, st, Z, args.warmup)
    t0 = time.perf_counter()
    st, Z, _, _ = oracle.steps(cfg, st, Z, args.steps)
    dt = time.perf_counter() - t0
    zones = w ** 3
    value = zones * args.steps / dt / 1e6
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"sweep_box recipe at {w}^3 (periodic; the {args.size}^3 workload's statistics), {args.steps} oracle "
              f"SSP-RK3 steps (after {args.warmup} warm-up), FP64, OpenMP over cells")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": f"{workload_name(args)}, timed on a {w}^3 sample of the same recipe per step",
                   "grid": [args.size] * 3, "zones": args.size ** 3, "sample_grid": [w] * 3,
                   "parallelism": "rank 0 only (host cores)", "sample": f"{w}^3 box of the same recipe per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu": cpu_description()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


OPS = load_op_counts() if os.path.exists(OP_COUNTS_PATH) else None


def totals_c2p_iters(pair):
    """Mean Newton iterations per inversion between two counter reads."""
    a, b = pair
    return (b["c2p_iters"] - a["c2p_iters"]) / max(b["c2p_calls"] - a["c2p_calls"], 1)


def run_ours(args, world, rank, local, dist):
    import numpy as np
    import torch
    from paper_1810_04597_gb300 import inputs, _lib
    from paper_1810_04597_gb300.echo import Solver

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    prob = inputs.sweep_box(args.size)
    n = prob.n
    zones = prob.ncells
    s = Solver(prob, precision=args.precision, device=str(dev))
    stream = s.stream
    s.set_prims()
    guess = args.guess if args.guess is not None else (4 if args.precision == 32 else 0)
    if guess & 1:
        # the network guess: train the default network first (untimed)
        from paper_1810_04597_gb300 import mlp
        state = mlp.default_network(device=str(dev), torus=True)[0]
        s.mlp_load(state)
    s.set_c2p_guess(guess)
    for _ in range(args.warmup):
        s.step()
    torch.cuda.synchronize()
    # the FP64 roofline peak: this GPU's rate on the library's FMA probe
    fp64_peak, fp64_src = measure_fp64_peak(dev)
    c_before = s.counters()

    # ---- timed region: K steps, device-resident inputs
    sampler = ClockSampler(gpu_index=None)
    sampler.start()
    time.sleep(0.3)
    s.profile(True)
    s.profile_read()
    barrier(dist)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        s.step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    ms = ev0.elapsed_time(ev1)
    prof = s.profile_read()
    s.profile(False)
    clocks = sampler.stop()
    ms_max = max_over_ranks(dist, ms)
    value = world * zones * args.steps / (ms_max * 1e-3) / 1e6
    c_after = s.counters()
    totals_run = (c_before, c_after)
    totals = s.reduce()
    fin64 = s.get_state() if (args.precision == 64 and not args.no_variants) else None

    # kernels launched in the timed region (a fill call launches 3 kernels,
    # the order-1 correction and its safeguard 6 each; the network's own pass
    # is a class of its own)
    per_call = {"fill_faces": 3, "fill_prims": 3, "correct": 6}
    launches = int(sum(cnt * per_call.get(k, 1) for k, (_, cnt) in prof.items()))

    # ---- roofline of the dominant kernel (live CUDA-event times)
    peaks, peak_src = load_peaks()
    timed = {k: v for k, v in prof.items() if k in KMODEL and v[1] > 0}
    dom = max(timed, key=lambda k: timed[k][0])
    dom_ms, dom_launches = timed[dom]
    avg_s = dom_ms / dom_launches * 1e-3
    units = kernel_units(dom, n)
    bytes_launch = units * kernel_bytes_per_unit(dom, args.precision)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_ctx = {"achieved": bytes_launch / avg_s / 1e9, "peak": hbm, "unit": "GB/s",
               "frac": bytes_launch / avg_s / 1e9 / hbm, "bytes_per_launch": bytes_launch,
               "peak_source": f"{peak_src} hbm_gbs" if peak_src == "measured" else "fallback 6800 GB/s"}
    share = {k: round(v[0] / ms, 4) for k, v in prof.items() if v[1] > 0}
    # whole-step HBM figure: the algorithmic bytes of every modelled kernel
    # launched in the timed region (each field read or written once per
    # launch) over the step time
    step_bytes = sum(kernel_units(k, n) * kernel_bytes_per_unit(k, args.precision) * v[1] for k, v in timed.items())
    hbm_step = {"bytes_per_zone_step": step_bytes / (zones * args.steps),
                "achieved_gbs": step_bytes / (ms * 1e-3) / 1e9,
                "frac": step_bytes / (ms * 1e-3) / 1e9 / hbm, "peak_gbs": hbm,
                "note": "algorithmic bytes of c2p, faces, EMFs and update per step / step time (fills and scalars "
                        "not counted)"}
    fl = FLOPS64[args.precision]
    if dom in fl:
        # bound by the FP64 pipe, not by HBM: the method's operations (the
        # oracle's count) per launch over the launch time, against the FP64
        # rate the probe measures on this GPU
        c_all = totals_c2p_iters(totals_run)
        alg = algorithmic_flops(OPS, dom, c_all)
        achieved = units * alg / avg_s / 1e12
        kernel_achieved = units * fl[dom] / avg_s / 1e12
        traffic = units * TRAFFIC_PER_FACE64 if (dom.startswith("faces") and args.precision == 64) else None
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": traffic, "peak_source": fp64_src,
                "flops_per_unit": alg, "flops_source": "the method's operations per unit, oracle counting build "
                                                       "(oracle/op_counts.json)",
                "units_per_launch": units,
                "kernel_flops_per_unit_ncu": fl[dom], "kernel_flops_frac": kernel_achieved / fp64_peak,
                "fp64_pipe_busy_ncu": FP64_PIPE_BUSY[args.precision].get(dom),
                "fp64_instr_frac": units * FP64_INSTR[args.precision][dom] / avg_s / FP64_PIPE_LANES_PER_S,
                "fp64_instr_frac_of": "the FP64 pipe's nominal lane rate (152 SMs x 2 per clock x 2.07 GHz)",
                "fp64_mix_cap_frac": fp64_mix_cap(fl[dom], FP64_INSTR[args.precision][dom], fp64_peak),
                "traffic_note": "dram bytes per face of a 128^3 ncu capture x faces per launch"
                if traffic is not None else "no ncu traffic figure for this kernel and precision",
                "avg_launch_ms": avg_s * 1e3, "hbm_context": hbm_ctx, "time_share": share}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": hbm_ctx["achieved"], "peak": hbm, "unit": "GB/s",
                "frac": hbm_ctx["frac"], "traffic": None, "peak_source": hbm_ctx["peak_source"],
                "bytes_per_launch": bytes_launch, "avg_launch_ms": avg_s * 1e3, "time_share": share}

    # ---- end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        nst = s.nstate
        # page-locked host buffers: the library's kernels read and write them
        # directly over the host link (no staging copy)
        st_host = torch.empty(nst, dtype=torch.float64, pin_memory=True)
        z_host = torch.empty(zones, dtype=torch.float64, pin_memory=True)
        out_host = torch.empty(nst, dtype=torch.float64, pin_memory=True)
        s.get_state(st_host)
        s.get_z(z_host)
        e2e_steps = max(1, min(args.steps, 5))
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            s.set_state(st_host, z_host)
            s.step()
            s.get_state(out_host)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        t_e2e = max_over_ranks(dist, t_e2e)
        e2e = {"value": world * zones * e2e_steps / t_e2e / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(st_host.numel() * 8 + z_host.numel() * 8),
               "d2h_bytes_per_step": int(out_host.numel() * 8), "steps": e2e_steps,
               "api": "echo_set_state(page-locked host) + echo_step + echo_get_state(page-locked host)"}

    # ---- FP32-bulk variant on the same input (timed the same way), and its
    #      relative L1 distance per field from the FP64 run after W + K steps
    variants = None
    if fin64 is not None:
        s32 = Solver(prob, precision=32, device=str(dev))
        s32.set_prims()
        s32.set_c2p_guess(4)
        for _ in range(args.warmup):
            s32.step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        s32.profile(True)
        s32.profile_read()
        e0.record(s32.stream)
        for _ in range(args.steps):
            s32.step()
        e1.record(s32.stream)
        torch.cuda.synchronize()
        ms32 = e0.elapsed_time(e1)
        prof32 = s32.profile_read()
        s32.profile(False)
        fin32 = s32.get_state()
        t32 = s32.reduce()
        N = zones
        bounds = [0, N, 2 * N, 3 * N, 4 * N, 5 * N]
        nx, ny, nz = n
        bounds += [5 * N + nz * ny * (nx + 1), 5 * N + nz * ny * (nx + 1) + nz * (ny + 1) * nx, len(fin64)]
        names = ["D", "S_x", "S_y", "S_z", "tau", "Bx", "By", "Bz"]
        l1 = {}
        for name, a, b in zip(names, bounds[:-1], bounds[1:]):
            den = float(np.sum(np.abs(fin64[a:b])))
            l1[name] = float(np.sum(np.abs(fin32[a:b] - fin64[a:b])) / den) if den > 0 else 0.0
        variants = {"fp32_bulk": {
            "value": world * zones * args.steps / (max_over_ranks(dist, ms32) * 1e-3) / 1e6, "unit": UNIT,
            "ms_per_step": ms32 / args.steps, "speedup_vs_fp64": ms / ms32,
            "l1_rel_vs_fp64_gpu": l1, "max_l1": max(l1.values()),
            "mean_newton_iters": t32["c2p_iters"] / max(t32["c2p_calls"], 1),
            "c2p_guess": "previous-stage Z refined by FP32 Newton steps; FP64 Newton judges",
            "roofline": fp32_c2p_roofline(prof32, ms32, zones, t32["c2p_iters"] / max(t32["c2p_calls"], 1),
                                          fp64_peak, fp64_src),
            "note": "FP32 storage/stencil, FP64 c2p and reductions; same input, same step count"}}
        del s32
        variants["fp64_high_order"] = run_order1_variant(args, prob, dev, world, dist, ms)
        variants["torus_256x128x128"] = run_torus_variant(args, dev, world, dist)
        mlp_state = None
        if not args.no_mlp:
            variants["fp32_mlp"], mlp_state = run_mlp_variant(args, prob, dev, world, dist, fin64, names, bounds,
                                                              ms)
            variants["c2p_guess_gain"] = run_guess_gain(prob, dev, mlp_state)
        if not args.no_sweep:
            variants["sweep_batch"] = run_sweep_variant(args, dev, world, dist, mlp_state)
        if not args.no_512 and mlp_state is not None:
            variants["box512_fp64_vs_fp32_mlp"] = run_box512_variant(args, dev, world, dist, mlp_state)

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_rows(args.cpu_budget)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == 64 else "f32 stencil + f64 c2p/reductions",
        "data": "synthetic (seeded sweep_box)",
        "config": {"workload": workload_name(args),
                   "grid": list(n), "zones": zones, "parallelism": f"replicas x{world}", "c2p_guess": guess,
                   "l2": "working set (~9 GB) larger than L2; no flush needed"},
        "clocks": clocks, "roofline": roof, "hbm_step": hbm_step, "cpu_baseline": cpu, "e2e": e2e,
        "variants": variants,
        "gpu_launches": launches,
        "check": {"c2p_fail": totals["c2p_fail"], "mean_newton_iters":
                  totals["c2p_iters"] / max(totals["c2p_calls"], 1), "dt_cfl": totals["dt_cfl"]},
    }
    return line if rank == 0 else None


def run_torus_variant(args, dev, world, dist, steps=50):
    """Fishbone-Moncrief torus on the Kerr metric (a = 0.9, beta = 100, 2 %
    pressure noise), 256 x 128 x 128 in (ln r, theta, phi) with atmosphere
    floors: FP32 bulk (guess: previous Z refined in FP32) and FP64 on the same
    input, W + 50 steps each; relative L1 per field of FP32 from FP64."""
    import numpy as np
    import torch
    from paper_1810_04597_gb300 import inputs
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.fm_torus((256, 128, 128), spin=0.9, beta=100.0)
    res = {"zones": prob.ncells, "steps": steps}
    fin = {}
    for prec in (64, 32):
        s = Solver(prob, precision=prec, device=str(dev))
        s.set_prims()
        if prec == 32:
            s.set_c2p_guess(4)
        for _ in range(args.warmup):
            s.step()
        torch.cuda.synchronize()
        c0 = s.counters()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(steps):
            s.step()
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(dist, e0.elapsed_time(e1))
        c1 = s.counters()
        calls = max(c1["c2p_calls"] - c0["c2p_calls"], 1)
        fin[prec] = s.get_state()
        res[f"fp{prec}"] = {"value": world * prob.ncells * steps / (ms * 1e-3) / 1e6, "unit": UNIT,
                            "ms_per_step": ms / steps,
                            "mean_newton_iters": (c1["c2p_iters"] - c0["c2p_iters"]) / calls,
                            "c2p_fail_per_call": (c1["c2p_fail"] - c0["c2p_fail"]) / calls,
                            "floor_hits_per_call": (c1["floor_hits"] - c0["floor_hits"]) / calls}
        s.close()
        del s
    N = prob.ncells
    a64, a32 = fin[64], fin[32]
    l1 = {}
    for q, name in enumerate(["D", "S_r", "S_theta", "S_phi", "tau"]):
        seg = slice(q * N, (q + 1) * N)
        den = float(np.sum(np.abs(a64[seg])))
        l1[name] = float(np.sum(np.abs(a32[seg] - a64[seg])) / den) if den > 0 else 0.0
    res["fp32"]["l1_rel_vs_fp64_gpu"] = l1
    res["fp32"]["l1_frame_vs_fp64_gpu"] = torus_frame_l1(prob, a64, a32)
    res["fp32"]["speedup_vs_fp64"] = res["fp64"]["ms_per_step"] / res["fp32"]["ms_per_step"]
    res["note"] = "Kerr-Schild, floors and fallbacks; FP32 bulk with FP64 c2p, metric and reductions"
    return res


def torus_frame_l1(prob, ref, got):
    """Relative L1 distances of the torus state `got` from `ref` that stay
    well conditioned where a component is near zero (S_theta in an
    equilibrium torus): D and tau as sum|d| / sum|ref|; each covariant
    momentum component in the local orthonormal frame,
    sum |dS_i| sqrt(gamma^ii) / sum |S| with |S| = sqrt(gamma^ij S_i S_j),
    the Kerr-Schild spatial metric at the cell centres (inputs.ks_metric_arrays)."""
    import numpy as np
    from paper_1810_04597_gb300 import inputs
    nx, ny, nz = prob.n
    N = nx * ny * nz
    x1 = prob.x0[0] + (np.arange(nx) + 0.5) * prob.dx[0]
    th = prob.x0[1] + (np.arange(ny) + 0.5) * prob.dx[1]
    X1, TH = np.meshgrid(x1, th)                       # (ny, nx)
    _, _, g11, g13, g22, g33 = inputs.ks_metric_arrays(X1, TH, prob.spin)
    det = g11 * g33 - g13 * g13
    gi11, gi22, gi33, gi13 = g33 / det, 1.0 / g22, g11 / det, -g13 / det
    cell = lambda st, q: st[q * N:(q + 1) * N].reshape(nz, ny, nx)
    S = [cell(ref, 1 + q) for q in range(3)]
    Smag = np.sqrt(gi11 * S[0] ** 2 + gi22 * S[1] ** 2 + gi33 * S[2] ** 2 + 2.0 * gi13 * S[0] * S[2])
    den = float(np.sum(Smag))
    out = {}
    for q, name in ((0, "D"), (4, "tau")):
        r = cell(ref, q)
        out[name] = float(np.sum(np.abs(cell(got, q) - r)) / max(float(np.sum(np.abs(r))), 1e-300))
    for q, (name, gii) in enumerate((("S_r", gi11), ("S_theta", gi22), ("S_phi", gi33))):
        out[name] = float(np.sum(np.abs(cell(got, 1 + q) - S[q]) * np.sqrt(gii)) / max(den, 1e-300))
    return out


def run_order1_variant(args, prob, dev, world, dist, ms64):
    """The same input and step count with the high-order form (order 1:
    point-value MP5, sixth-order cell-centre B, flux-derivative correction
    of the fluxes and EMFs), FP64."""
    import dataclasses
    import torch
    from paper_1810_04597_gb300.echo import Solver
    p1 = dataclasses.replace(prob, order=1)
    s = Solver(p1, precision=64, device=str(dev))
    s.set_prims()
    for _ in range(args.warmup):
        s.step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    for _ in range(args.steps):
        s.step()
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1)
    t = s.reduce()
    del s
    return {"value": world * prob.ncells * args.steps / (max_over_ranks(dist, ms1) * 1e-3) / 1e6, "unit": UNIT,
            "ms_per_step": ms1 / args.steps, "cost_vs_order0": ms1 / ms64, "c2p_fail": t["c2p_fail"],
            "note": "FP64, high-order form (flux-derivative correction), same input and steps"}


def run_mlp_variant(args, prob, dev, world, dist, fin64, names, bounds, ms64):
    """FP32 bulk with the c2p-guess network: train the network on FP64 runs
    of the 128^3 periodic boxes and of four tori (untimed), then time W + K
    steps on the workload from the same input as the FP64 run."""
    import numpy as np
    import torch
    from paper_1810_04597_gb300 import mlp
    from paper_1810_04597_gb300.echo import Solver
    t0 = time.perf_counter()
    state, losses, _, (Xte, Yte) = mlp.default_network(device=str(dev), torus=True)
    err = mlp.guess_error(state, Xte, Yte).cpu().numpy()
    err_tc = mlp.guess_error(state, Xte, Yte, tensor_cores=True).cpu().numpy()
    t_train = time.perf_counter() - t0
    s = Solver(prob, precision=32, device=str(dev))
    s.set_prims()
    s.mlp_load(state)
    s.set_c2p_guess(5)
    for _ in range(args.warmup):
        s.step()
    torch.cuda.synchronize()
    c0 = s.counters()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    for _ in range(args.steps):
        s.step()
    e1.record(s.stream)
    torch.cuda.synchronize()
    msm = e0.elapsed_time(e1)
    c1 = s.counters()
    fin = s.get_state()
    l1 = {}
    for name, a, b in zip(names, bounds[:-1], bounds[1:]):
        den = float(np.sum(np.abs(fin64[a:b])))
        l1[name] = float(np.sum(np.abs(fin[a:b] - fin64[a:b])) / den) if den > 0 else 0.0
    calls = max(c1["c2p_calls"] - c0["c2p_calls"], 1)
    out = {"value": world * prob.ncells * args.steps / (max_over_ranks(dist, msm) * 1e-3) / 1e6, "unit": UNIT,
           "ms_per_step": msm / args.steps, "speedup_vs_fp64": ms64 / msm,
           "l1_rel_vs_fp64_gpu": l1, "max_l1": max(l1.values()),
           "mean_newton_iters": (c1["c2p_iters"] - c0["c2p_iters"]) / calls,
           "mlp_fallback_per_call": (c1["mlp_fallback"] - c0["mlp_fallback"]) / calls,
           "guess_rel_err_median_heldout": float(np.median(err)),
           "guess_rel_err_p99_heldout": float(np.quantile(err, 0.99)),
           "guess_rel_err_median_heldout_tensor_cores": float(np.median(err_tc)),
           "guess_rel_err_p99_heldout_tensor_cores": float(np.quantile(err_tc, 0.99)),
           "train_seconds": t_train, "train_final_loss": float(losses[-50:].mean().item()),
           "c2p_guess": "network (trained on the GPU, untimed) refined by FP32 Newton steps; FP64 Newton judges",
           "note": "FP32 bulk"}
    del s
    return out, state


def fp32_c2p_roofline(prof, ms, zones, newton_iters, fp64_peak, fp64_src):
    """The FP32-bulk path's dominant kernel is c2p, bound by the FP64 pipe:
    the method's FP64 operations per cell (the oracle's count at the FP64
    Newton iterations this path takes; its FP32 refinement is not counted)
    x cells per launch / its live CUDA-event launch time, against the
    measured FP64 peak; the kernel's own ncu count beside it."""
    c_ms, c_n = prof["c2p"]
    avg_s = c_ms / max(c_n, 1) * 1e-3
    alg = algorithmic_flops(OPS, "c2p", newton_iters)
    achieved = zones * alg / avg_s / 1e12
    return {"kernel": "c2p", "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak, "peak_source": fp64_src, "flops_per_unit": alg,
            "flops_source": "the method's FP64 operations per cell at %.2f FP64 Newton iterations, oracle counting "
                            "build (oracle/op_counts.json); the judging step's f' among them comes from the FP32 "
                            "refinement" % newton_iters,
            "units_per_launch": zones,
            "kernel_flops_per_unit_ncu": FLOPS64[32]["c2p"],
            "kernel_flops_frac": zones * FLOPS64[32]["c2p"] / avg_s / 1e12 / fp64_peak,
            "fp64_pipe_busy_ncu": FP64_PIPE_BUSY[32]["c2p"], "avg_launch_ms": avg_s * 1e3,
            "fp64_instr_frac": zones * FP64_INSTR[32]["c2p"] / avg_s / FP64_PIPE_LANES_PER_S,
            "fp64_instr_frac_of": "the FP64 pipe's nominal lane rate (152 SMs x 2 per clock x 2.07 GHz)",
            "fp64_mix_cap_frac": fp64_mix_cap(FLOPS64[32]["c2p"], FP64_INSTR[32]["c2p"], fp64_peak),
            "time_share": {k: round(v[0] / ms, 4) for k, v in prof.items() if v[1] > 0}}


def run_guess_gain(prob, dev, mlp_state, warm=2, steps=3):
    """What the network guess gains: the workload's c2p with the previous-
    stage Z, the network (tensor cores) and the cold guess as start, in FP64
    (plain Newton from the guess) and in the FP32-bulk form (guess refined in
    FP32, one FP64 judging step): c2p kernel time per call (the library's
    per-kernel CUDA events), mean and 99th-percentile Newton iterations per
    inversion (from the iteration histogram), network restarts.  Each guess
    runs `steps` steps from the same state (`warm` steps with the previous-Z
    guess first)."""
    import numpy as np
    import torch
    from paper_1810_04597_gb300.echo import Solver
    out = {}
    for prec, modes in ((64, {"previous": 0, "network": 1, "network_inside_c2p": 17, "cold": 2}),
                        (32, {"previous": 4, "network": 5, "network_inside_c2p": 21, "cold": 6})):
        res = {}
        for name, mode in modes.items():
            s = Solver(prob, precision=prec, device=str(dev))
            s.set_prims()
            s.mlp_load(mlp_state)
            if prec == 32:
                s.set_c2p_guess(4)
            for _ in range(warm):
                s.step()
            s.set_c2p_guess(mode)
            torch.cuda.synchronize()
            c0 = s.counters()
            s.profile(True)
            s.profile_read()
            for _ in range(steps):
                s.step()
            prof = s.profile_read()
            s.profile(False)
            c1 = s.counters()
            calls = max(c1["c2p_calls"] - c0["c2p_calls"], 1)
            h = np.array(c1["c2p_iter_hist"]) - np.array(c0["c2p_iter_hist"])
            cum = np.cumsum(h) / max(int(h.sum()), 1)
            ms, nl = prof["c2p"]
            ms += prof["network"][0]   # the network's own pass, per c2p call
            res[name] = {"c2p_ms_per_call": ms / max(nl, 1),
                         "network_pass_ms_per_call": prof["network"][0] / max(nl, 1),
                         "mean_newton_iters": (c1["c2p_iters"] - c0["c2p_iters"]) / calls,
                         "p99_newton_iters": int(np.searchsorted(cum, 0.99)),
                         "mlp_fallback_per_call": (c1["mlp_fallback"] - c0["mlp_fallback"]) / calls,
                         "network_starts_per_call": (c1["mlp_used"] - c0["mlp_used"]) / calls}
            del s
        # a cold restart (state without its Newton memory): one inversion
        for name, mode in (("restart_cold", modes["cold"]), ("restart_network", modes["network"])):
            s = Solver(prob, precision=prec, device=str(dev))
            s.set_prims()
            s.mlp_load(mlp_state)
            for _ in range(warm):
                s.step()
            s.set_state(s.get_state())
            c0 = s.counters()
            s.profile(True)
            s.profile_read()
            s.c2p(mode, stats=False)
            prof = s.profile_read()
            s.profile(False)
            c1 = s.counters()
            calls = max(c1["c2p_calls"] - c0["c2p_calls"], 1)
            ms, nl = prof["c2p"]
            ms += prof["network"][0]
            res[name] = {"c2p_ms_per_call": ms / max(nl, 1),
                         "network_pass_ms_per_call": prof["network"][0] / max(nl, 1),
                         "mean_newton_iters": (c1["c2p_iters"] - c0["c2p_iters"]) / calls,
                         "mlp_fallback_per_call": (c1["mlp_fallback"] - c0["mlp_fallback"]) / calls,
                         "network_starts_per_call": (c1["mlp_used"] - c0["mlp_used"]) / calls}
            del s
        out[f"fp{prec}"] = res
    # the torus atmosphere (held-out torus, FP64, 6 steps): the previous-stage
    # Z against the per-cell choice
    from paper_1810_04597_gb300 import inputs
    tprob = inputs.fm_torus((96, 48, 48), spin=0.5, beta=30.0, seed=inputs.SEED_BASE + 299)
    res = {}
    for name, mode in (("previous", 0), ("network", 1)):
        s = Solver(tprob, precision=64, device=str(dev))
        s.set_prims()
        s.mlp_load(mlp_state)
        s.set_c2p_guess(mode)
        c0 = s.counters()
        s.profile(True)
        s.profile_read()
        for _ in range(6):
            s.step()
        prof = s.profile_read()
        s.profile(False)
        c1 = s.counters()
        calls = max(c1["c2p_calls"] - c0["c2p_calls"], 1)
        ms, nl = prof["c2p"]
        ms += prof["network"][0]
        res[name] = {"c2p_ms_per_call": ms / max(nl, 1),
                     "network_pass_ms_per_call": prof["network"][0] / max(nl, 1),
                     "mean_newton_iters": (c1["c2p_iters"] - c0["c2p_iters"]) / calls,
                     "mlp_fallback_per_call": (c1["mlp_fallback"] - c0["mlp_fallback"]) / calls,
                     "network_starts_per_call": (c1["mlp_used"] - c0["mlp_used"]) / calls,
                     "c2p_fail_per_call": (c1["c2p_fail"] - c0["c2p_fail"]) / calls}
        del s
    out["torus_fp64"] = res
    out["note"] = ("c2p on the workload from each start: FP64 plain Newton, FP32 bulk with FP32 refinement and "
                   "one FP64 judging step; iterations are FP64 Newton iterations (network attempt and restart "
                   "together); the previous-stage Z is the plain method's guess; network: per-cell choice "
                   "between the network start and the previous Z (tensor-core pass over the listed cells, "
                   "then the c2p kernel); network_inside_c2p: the same choice with the network fused into the "
                   "c2p kernel; restart_*: one inversion of the state without its Newton memory; torus_fp64: "
                   "a held-out 96x48x48 torus (spin 0.5, beta 30), 6 steps")
    return out


def run_box512_variant(args, dev, world, dist, mlp_state):
    """The 512^3 periodic box of the parity recipe (smooth_box): FP64 and FP32
    bulk + network c2p guess (tensor cores) on the same input, W + K steps
    each, and the relative L1 distance per field of the FP32 + network state
    from the FP64 state."""
    import numpy as np
    import torch
    from paper_1810_04597_gb300 import inputs
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.smooth_box(512)
    out = {"zones": prob.ncells, "steps": args.steps}

    def timed(s):
        for _ in range(args.warmup):
            s.step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(args.steps):
            s.step()
        e1.record(s.stream)
        torch.cuda.synchronize()
        return max_over_ranks(dist, e0.elapsed_time(e1))

    s = Solver(prob, precision=64, device=str(dev))
    s.set_prims()
    ms64 = timed(s)
    fin64 = s.get_state()
    s.close()
    del s
    s = Solver(prob, precision=32, device=str(dev))
    s.set_prims()
    s.mlp_load(mlp_state)
    s.set_c2p_guess(5)
    c0 = s.counters()
    ms32 = timed(s)
    c1 = s.counters()
    fin32 = s.get_state()
    s.close()
    del s
    N = prob.ncells
    nx, ny, nz = prob.n
    bounds = [0, N, 2 * N, 3 * N, 4 * N, 5 * N, 5 * N + nz * ny * (nx + 1),
              5 * N + nz * ny * (nx + 1) + nz * (ny + 1) * nx, len(fin64)]
    names = ["D", "S_x", "S_y", "S_z", "tau", "Bx", "By", "Bz"]
    l1 = {}
    for name, a, b in zip(names, bounds[:-1], bounds[1:]):
        den = float(np.sum(np.abs(fin64[a:b])))
        l1[name] = float(np.sum(np.abs(fin32[a:b] - fin64[a:b])) / den) if den > 0 else 0.0
    calls = max(c1["c2p_calls"] - c0["c2p_calls"], 1)
    out.update({
        "fp64": {"value": world * N * args.steps / (ms64 * 1e-3) / 1e6, "unit": UNIT,
                 "ms_per_step": ms64 / args.steps},
        "fp32_mlp": {"value": world * N * args.steps / (ms32 * 1e-3) / 1e6, "unit": UNIT,
                     "ms_per_step": ms32 / args.steps, "speedup_vs_fp64": ms64 / ms32,
                     "l1_rel_vs_fp64_gpu": l1, "max_l1": max(l1.values()),
                     "mean_newton_iters": (c1["c2p_iters"] - c0["c2p_iters"]) / calls,
                     "mlp_fallback_per_call": (c1["mlp_fallback"] - c0["mlp_fallback"]) / calls},
        "note": "smooth_box recipe at 512^3 (|k| <= 3 modes), same input and step count for both"})
    return out


def run_sweep_variant(args, dev, world, dist, mlp_state):
    """The 16-run Fishbone-Moncrief torus sweep (uneven sizes 64x32x32 ..
    192x96x96, spins 0..0.98, beta 10/100), FP32 bulk + network c2p guess,
    advanced as one batch (schedule and tiles autotuned over persistent
    cooperative, per-phase and run-major, replayed from one CUDA graph) and,
    for comparison, one run at a time without a graph."""
    import torch
    from paper_1810_04597_gb300.batch import MODE_NAMES, Batch, autotune, sweep_runs

    def make():
        sol = sweep_runs(precision=32, device=str(dev))
        for x in sol:
            if mlp_state is not None:
                x.mlp_load(mlp_state)
                x.set_c2p_guess(5)
            else:
                x.set_c2p_guess(4)
        return sol

    sol = make()
    zones = sum(x.ncells for x in sol)
    b = Batch(sol)
    tune = autotune(b, reps=2, cache=False, graph=True)
    for _ in range(args.warmup):
        b.step()
    torch.cuda.synchronize()
    c0 = [x.counters() for x in sol]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    for _ in range(args.steps):
        b.step()
    e1.record(b.stream)
    torch.cuda.synchronize()
    msb = e0.elapsed_time(e1)
    c1 = [x.counters() for x in sol]
    calls = sum(y["c2p_calls"] - x["c2p_calls"] for x, y in zip(c0, c1))
    fb = sum(y["mlp_fallback"] - x["mlp_fallback"] for x, y in zip(c0, c1))
    fl = sum(y["floor_hits"] - x["floor_hits"] for x, y in zip(c0, c1))
    its = sum(y["c2p_iters"] - x["c2p_iters"] for x, y in zip(c0, c1))
    b.close()
    del sol
    # the same sweep, one run at a time (a launch sequence per run and stage)
    sol = make()
    for _ in range(args.warmup):
        for x in sol:
            x.step()
    torch.cuda.synchronize()
    e0.record(torch.cuda.current_stream())
    for _ in range(args.steps):
        for x in sol:
            x.step()
    e1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    mss = e0.elapsed_time(e1)
    del sol
    return {"value": world * zones * args.steps / (max_over_ranks(dist, msb) * 1e-3) / 1e6, "unit": UNIT,
            "zones": zones, "runs": 16, "ms_per_step": msb / args.steps,
            "one_at_a_time_value": zones * args.steps / (mss * 1e-3) / 1e6,
            "batch_speedup": mss / msb,
            "autotune": {"best": {k: tune[k] for k in ("mode", "tile", "blocks_per_sm", "dynamic", "branches", "ms")},
                         "best_per_mode_ms": {MODE_NAMES[m]: min(c["ms"] for c in tune["candidates"] if c["mode"] == m)
                                              for m in MODE_NAMES}},
            "mean_newton_iters": its / max(calls, 1), "mlp_fallback_per_call": fb / max(calls, 1),
            "floor_hits_per_call": fl / max(calls, 1),
            "note": "FP32 bulk + network c2p guess, per-run CFL dt, whole step replayed from one CUDA graph"}



def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--precision", type=int, default=64, choices=(32, 64))
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-mlp", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-512", action="store_true", help="skip the 512^3 FP64 / FP32 + network variant")
    ap.add_argument("--guess", type=int, default=None, choices=(0, 1, 2, 4, 5, 6, 9, 13, 17, 21),
                    help="c2p guess mode of the main line (default: 0 for FP64, 4 for FP32)")
    args = ap.parse_args()
    world, rank, local = dist_info()
    if args.impl == "reference":
        line = run_reference(args, world, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0
    dist = init_dist(world, local)
    line = run_ours(args, world, rank, local, dist)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
