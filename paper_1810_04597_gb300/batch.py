"""A batch of independent runs advanced by one persistent cooperative kernel
per SSP-RK3 stage (see ``echo_batch_*`` in include/echo.h), and the tile
autotuner.  Torch supplies the batch workspace and the stream only."""
from __future__ import annotations

import json
import os

from . import _lib, inputs
from .echo import Solver

_HERE = os.path.dirname(os.path.abspath(__file__))
TUNE_CACHE = os.path.join(_HERE, "_build", "batch_autotune.json")


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

    def configure(self, tile=256, blocks_per_sm=None, dynamic=True):
        mb = _lib.echo_batch_max_blocks_per_sm(self.b)
        bps = mb if blocks_per_sm is None else min(blocks_per_sm, mb)
        _lib.echo_batch_config(self.b, tile, bps, 1 if dynamic else 0)
        self.config = dict(tile=tile, blocks_per_sm=bps, dynamic=bool(dynamic))

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


def autotune(batch: Batch, tiles=(128, 256, 512, 1024), queue=(True, False), reps=2, key=None, cache=True):
    """Time `reps` steps for every (tile, blocks per SM, queue kind) and keep
    the fastest; the choice is cached per device and batch signature.  The
    runs' states advance while tuning."""
    import torch
    mb = _lib.echo_batch_max_blocks_per_sm(batch.b)
    bpss = sorted({mb, max(1, mb // 2)})
    dev = torch.cuda.get_device_name(batch.solvers[0].device)
    sig = key or "|".join("x".join(str(v) for v in s.problem.n) for s in batch.solvers)
    ck = f"{dev}|p{batch.solvers[0].precision}|{sig}"
    if cache and os.path.exists(TUNE_CACHE):
        try:
            db = json.load(open(TUNE_CACHE))
            if ck in db:
                c = db[ck]
                batch.configure(c["tile"], c["blocks_per_sm"], c["dynamic"])
                return dict(c, cached=True)
        except Exception:
            pass
    best = None
    results = []
    for tile in tiles:
        for bps in bpss:
            for dyn in queue:
                batch.configure(tile, bps, dyn)
                batch.step()                       # warm
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(batch.stream)
                for _ in range(reps):
                    batch.step()
                e1.record(batch.stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                results.append(dict(tile=tile, blocks_per_sm=bps, dynamic=dyn, ms=ms))
                if best is None or ms < best["ms"]:
                    best = results[-1]
    batch.configure(best["tile"], best["blocks_per_sm"], best["dynamic"])
    out = dict(best, cached=False, candidates=results)
    if cache:
        os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
        db = {}
        if os.path.exists(TUNE_CACHE):
            try:
                db = json.load(open(TUNE_CACHE))
            except Exception:
                db = {}
        db[ck] = {k: best[k] for k in ("tile", "blocks_per_sm", "dynamic", "ms")}
        json.dump(db, open(TUNE_CACHE, "w"), indent=1)
    return out
