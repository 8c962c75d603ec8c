"""A batch of independent runs advanced together (see ``echo_batch_*`` in
include/echo.h) under one of three schedules -- one persistent cooperative
kernel per SSP-RK3 stage, one launch per phase over all runs, or each run's
own launch sequence in turn -- optionally replayed from one CUDA graph, and
the autotuner that picks the schedule and its tiles.  Torch supplies the
batch workspace and the stream only."""
from __future__ import annotations

import json
import os

from . import _lib, inputs
from .echo import Solver

_HERE = os.path.dirname(os.path.abspath(__file__))
TUNE_CACHE = os.path.join(_HERE, "_build", "batch_autotune.json")

PERSISTENT, PHASED, RUN_MAJOR = 0, 1, 2
MODE_NAMES = {PERSISTENT: "persistent", PHASED: "phased", RUN_MAJOR: "run_major"}


class Batch:
    def __init__(self, solvers, stream=None):
        import torch
        self.solvers = list(solvers)
        dev = self.solvers[0].device
        self.b = _lib.echo_batch_create([s.ctx for s in self.solvers])
        nbytes = _lib.echo_batch_workspace_bytes(self.b)
        with torch.cuda.device(dev):
            # a created stream (graph capture is impossible on the legacy one);
            # steps are ordered against the caller's current stream by events
            self.stream = stream if stream is not None else torch.cuda.Stream(dev)
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            self.stream.wait_stream(torch.cuda.current_stream(dev))
            _lib.echo_batch_bind(self.b, self.ws.data_ptr(), nbytes, self.stream.cuda_stream)
        self.device = dev
        self.config = None

    @property
    def zones(self) -> int:
        return sum(s.ncells for s in self.solvers)

    def configure(self, tile=256, blocks_per_sm=None, dynamic=True, mode=PERSISTENT, branches=1):
        """`mode`: PERSISTENT, PHASED or RUN_MAJOR; tile, blocks per SM and the
        queue kind apply to the first two, `branches` (concurrent streams) to
        RUN_MAJOR."""
        import torch
        mb = _lib.echo_batch_max_blocks_per_sm(self.b)
        bps = mb if blocks_per_sm is None else min(blocks_per_sm, mb)
        _lib.echo_batch_config(self.b, tile, bps, 1 if dynamic else 0)
        _lib.echo_batch_mode(self.b, int(mode))
        with torch.cuda.device(self.device):
            _lib.echo_batch_branches(self.b, min(int(branches), len(self.solvers)))
        self.config = dict(tile=tile, blocks_per_sm=bps, dynamic=bool(dynamic), mode=MODE_NAMES[int(mode)],
                           branches=int(branches))

    def graph(self, enable=True):
        _lib.echo_batch_graph(self.b, enable)

    def step(self, dt=0.0):
        import torch
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        _lib.echo_batch_step(self.b, dt)
        cur.wait_stream(self.stream)

    def close(self):
        if getattr(self, "b", None):
            _lib.echo_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sweep_runs(scale=1, precision=32, device="cuda:0", steps=100):
    """The 16-run torus parameter sweep: run i has size index i // 4 in
    (64x32x32, 96x48x48, 128x64x64, 192x96x96) / scale, spin
    (0, 0.5, 0.9, 0.98)[i % 4], beta 10 if (i // 4 + i % 4) is even else 100."""
    sizes = [(64, 32, 32), (96, 48, 48), (128, 64, 64), (192, 96, 96)]
    spins = [0.0, 0.5, 0.9, 0.98]
    sol = []
    for i in range(16):
        n = tuple(max(8, v // scale) for v in sizes[i // 4])
        beta = 10.0 if (i // 4 + i % 4) % 2 == 0 else 100.0
        prob = inputs.fm_torus(n, spin=spins[i % 4], beta=beta, seed=inputs.SEED_BASE + 50 + i, steps=steps)
        s = Solver(prob, precision=precision, device=device)
        s.set_prims()
        sol.append(s)
    return sol


def candidates(runs: int, max_blocks_per_sm: int, tiles=(128, 256, 512, 1024), queue=(True, False),
               high_order: bool = False):
    """The schedules the autotuner times, as (tile, blocks per SM, dynamic
    queue, mode, branches): persistent with each tile, blocks-per-SM choice
    and queue kind, per-phase with each tile (both for the form of order 0
    only), and run-major with 1, 2, 4, 8 and all-runs graph branches (never
    more branches than runs)."""
    mb = max_blocks_per_sm
    bpss = sorted({mb, max(1, mb // 2), min(mb, 2), min(mb, 3)})
    cands = []
    if not high_order:
        cands += [(tile, bps, dyn, PERSISTENT, 1) for tile in tiles for bps in bpss for dyn in queue]
        cands += [(tile, mb, True, PHASED, 1) for tile in tiles]
    cands += [(256, mb, True, RUN_MAJOR, k) for k in sorted({1, 2, 4, 8, runs}) if k <= runs]
    return cands


def _load_cache():
    try:
        with open(TUNE_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune(batch: Batch, tiles=(128, 256, 512, 1024), queue=(True, False), reps=2, key=None, cache=True,
             graph=True):
    """Time `reps` steps (replayed from a graph when `graph`) for every
    schedule -- persistent with each (tile, blocks per SM, queue kind), phased
    with each tile, run-major -- and keep the fastest; the choice is cached
    per device and batch signature.  The runs' states advance while tuning."""
    import torch
    mb = _lib.echo_batch_max_blocks_per_sm(batch.b)
    dev = torch.cuda.get_device_name(batch.solvers[0].device)
    sig = key or "|".join("x".join(str(v) for v in s.problem.n) for s in batch.solvers)
    ck = f"{dev}|p{batch.solvers[0].precision}|g{int(graph)}|{sig}"
    if cache:
        c = _load_cache().get(ck)
        if c is not None:
            batch.configure(c["tile"], c["blocks_per_sm"], c["dynamic"], c["mode"], c["branches"])
            batch.graph(graph)
            return dict(c, cached=True)
    best = None
    results = []
    # the persistent and per-phase schedules run the form of order 0 only
    high = any(getattr(s.problem, "order", 0) for s in batch.solvers)
    cands = candidates(len(batch.solvers), mb, tiles, queue, high)
    batch.graph(graph)
    for tile, bps, dyn, mode, br in cands:
        batch.configure(tile, bps, dyn, mode, br)
        batch.step()                       # warm (and capture)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(batch.stream)
        for _ in range(reps):
            batch.step()
        e1.record(batch.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        results.append(dict(tile=tile, blocks_per_sm=bps, dynamic=dyn, mode=mode, branches=br, ms=ms))
        if best is None or ms < best["ms"]:
            best = results[-1]
    batch.configure(best["tile"], best["blocks_per_sm"], best["dynamic"], best["mode"], best["branches"])
    out = dict(best, cached=False, candidates=results)
    if cache:
        os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
        db = _load_cache()
        db[ck] = {k: best[k] for k in ("tile", "blocks_per_sm", "dynamic", "mode", "branches", "ms")}
        with open(TUNE_CACHE, "w") as f:
            json.dump(db, f, indent=1)
    return out
