"""User-facing wrapper: one GRMHD grid on one GPU.

PyTorch supplies the device workspace and the CUDA stream and nothing else;
every operation on the state runs in the library's kernels through the C ABI
(``_lib``).  Without the CUDA library or a GPU the constructor raises --
there is no CPU path.
"""
from __future__ import annotations

import numpy as np

from . import _lib


class Solver:
    """A context bound to a torch-allocated workspace on ``device``.

    ``problem`` is any object with the attributes of ``inputs.Problem``
    (grid, boundary kinds, metric, EOS and CFL number); ``precision`` is 64
    (FP64 throughout) or 32 (FP32 storage and stencil, FP64 c2p/reductions).
    """

    def __init__(self, problem, precision: int = 64, device: str = "cuda:0", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1810_04597_gb300.Solver needs a CUDA GPU")
        self.device = torch.device(device)
        self.problem = problem
        g = _lib.echo_grid()
        for d in range(3):
            g.n[d] = int(problem.n[d])
            g.x0[d] = float(problem.x0[d])
            g.dx[d] = float(problem.dx[d])
        for s in range(6):
            g.bc[s] = int(problem.bc[s])
        m = _lib.echo_metric(int(problem.metric), float(problem.spin))
        e = _lib.echo_eos(float(problem.gamma), int(bool(problem.floors)), float(problem.rho_floor),
                          float(problem.rho_floor_pow), float(problem.p_floor), float(problem.p_floor_pow))
        self.precision = int(precision)
        self.ctx = _lib.echo_init(g, m, e, self.precision, float(problem.cfl))
        if getattr(problem, "order", 0):
            _lib.echo_set_order(self.ctx, int(problem.order))
        self.nbytes = _lib.echo_workspace_bytes(self.ctx)
        self.nstate = _lib.echo_state_count(self.ctx)
        self.ncells = int(problem.n[0]) * int(problem.n[1]) * int(problem.n[2])
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
            _lib.echo_bind(self.ctx, self.workspace.data_ptr(), self.nbytes, self.stream.cuda_stream)

    # -- state in / out
    def set_prims(self, prims5=None, bface=None):
        prims5 = self.problem.prims if prims5 is None else prims5
        bface = self.problem.bface if bface is None else bface
        if isinstance(prims5, np.ndarray):
            prims5 = np.ascontiguousarray(prims5, dtype=np.float64)
            bface = np.ascontiguousarray(bface, dtype=np.float64)
        _lib.echo_set_prims(self.ctx, prims5, bface)

    def set_state(self, state, Z=None):
        _lib.echo_set_state(self.ctx, state, Z)

    def get_state(self, out=None):
        out = np.empty(self.nstate) if out is None else out
        return _lib.echo_get_state(self.ctx, out)

    def get_prims(self, out=None):
        out = np.empty(8 * self.ncells) if out is None else out
        _lib.echo_get_prims(self.ctx, out)
        return out.reshape(8, -1) if isinstance(out, np.ndarray) else out

    def get_z(self, out=None):
        out = np.empty(self.ncells) if out is None else out
        return _lib.echo_get_z(self.ctx, out)

    # -- operations
    def c2p(self, guess_mode: int = 0, stats: bool = True):
        t = _lib.echo_totals() if stats else None
        _lib.echo_c2p(self.ctx, guess_mode, t)
        return t.as_dict() if stats else None

    def rhs(self, out=None):
        out = np.empty(self.nstate) if out is None else out
        return _lib.echo_rhs(self.ctx, out)

    def step(self, dt: float = 0.0):
        _lib.echo_step(self.ctx, dt)

    def reduce(self) -> dict:
        return _lib.echo_reduce(self.ctx).as_dict()

    def counters(self) -> dict:
        return _lib.echo_counters(self.ctx).as_dict()

    def mlp_load(self, state):
        _lib.echo_mlp_load(self.ctx, state)

    def set_c2p_guess(self, mode: int):
        _lib.echo_set_c2p_guess(self.ctx, mode)

    def mlp_dataset(self, X, Y, offset: int = 0, stride: int = 1):
        _lib.echo_mlp_dataset(self.ctx, X, Y, X.shape[0], offset, stride)

    def profile(self, enable: bool = True):
        _lib.echo_profile(self.ctx, enable)

    def profile_read(self) -> dict:
        return _lib.echo_profile_read(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            _lib.echo_destroy(self.ctx)
            self.ctx = None
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
