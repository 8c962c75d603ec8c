"""ctypes binding of ``include/echo.h`` -- argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic on the state.  Array arguments may be NumPy arrays (host memory,
FP64, C-contiguous) or torch CUDA tensors (device memory, FP64); the
``on_device`` flag of the C call is derived from the argument.  A non-zero
status raises :class:`EchoError` with the library's message.

The library is ``_build/libecho.so`` next to this file (see ``build.py``).
There is no fallback: if it is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ECHO_OK = 0
ECHO_EINVAL = -1
ECHO_ECUDA = -2
ECHO_ENOMEM = -3
ECHO_EC2P = -4
ECHO_ETIMEOUT = -5
ECHO_ESTATE = -6
ECHO_ERANGE = -7
ECHO_STATIC_MAX_ROWS = 65536
ECHO_C2P_HIST = 16
_NAMES = {0: "ECHO_OK", -1: "ECHO_EINVAL", -2: "ECHO_ECUDA", -3: "ECHO_ENOMEM", -4: "ECHO_EC2P",
          -5: "ECHO_ETIMEOUT", -6: "ECHO_ESTATE", -7: "ECHO_ERANGE"}

BC_PERIODIC, BC_OUTFLOW, BC_AXIS = 0, 1, 2
METRIC_FLAT, METRIC_KERR_SCHILD = 0, 1


class EchoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class echo_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("x0", ctypes.c_double * 3), ("dx", ctypes.c_double * 3),
                ("bc", ctypes.c_int * 6)]


class echo_metric(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("spin", ctypes.c_double)]


class echo_eos(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("floors", ctypes.c_int), ("rho_floor", ctypes.c_double),
                ("rho_floor_pow", ctypes.c_double), ("p_floor", ctypes.c_double),
                ("p_floor_pow", ctypes.c_double)]


class echo_totals(ctypes.Structure):
    _fields_ = [("dt_cfl", ctypes.c_double), ("mass", ctypes.c_double), ("energy", ctypes.c_double),
                ("mom", ctypes.c_double * 3), ("max_divb", ctypes.c_double),
                ("c2p_iters", ctypes.c_longlong), ("c2p_calls", ctypes.c_longlong),
                ("c2p_fail", ctypes.c_longlong), ("floor_hits", ctypes.c_longlong),
                ("fallback_faces", ctypes.c_longlong), ("mlp_fallback", ctypes.c_longlong),
                ("c2p_iter_hist", ctypes.c_longlong * ECHO_C2P_HIST), ("mlp_used", ctypes.c_longlong),
                ("guard_faces", ctypes.c_longlong)]

    def as_dict(self):
        return dict(dt_cfl=self.dt_cfl, mass=self.mass, energy=self.energy, mom=list(self.mom),
                    max_divb=self.max_divb, c2p_iters=self.c2p_iters, c2p_calls=self.c2p_calls,
                    c2p_fail=self.c2p_fail, floor_hits=self.floor_hits,
                    fallback_faces=self.fallback_faces, mlp_fallback=self.mlp_fallback,
                    c2p_iter_hist=list(self.c2p_iter_hist), mlp_used=self.mlp_used,
                    guard_faces=self.guard_faces)


# Exported entry points and their C signatures.
_P = ctypes.c_void_p
_SIGS = {
    "echo_init": (ctypes.c_int, [ctypes.POINTER(echo_grid), ctypes.POINTER(echo_metric),
                                 ctypes.POINTER(echo_eos), ctypes.c_int, ctypes.c_double,
                                 ctypes.POINTER(_P)]),
    "echo_set_order": (ctypes.c_int, [_P, ctypes.c_int]),
    "echo_workspace_bytes": (ctypes.c_size_t, [_P]),
    "echo_state_count": (ctypes.c_size_t, [_P]),
    "echo_bind": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "echo_set_prims": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "echo_set_state": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "echo_get_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "echo_get_prims": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "echo_get_z": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "echo_c2p": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(echo_totals)]),
    "echo_rhs": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "echo_step": (ctypes.c_int, [_P, ctypes.c_double]),
    "echo_reduce": (ctypes.c_int, [_P, ctypes.POINTER(echo_totals)]),
    "echo_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "echo_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]),
    "echo_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
    "echo_counters": (ctypes.c_int, [_P, ctypes.POINTER(echo_totals)]),
    "echo_selftest_conversions": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_ulonglong, _P, _P]),
    "echo_selftest_recip": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_ulonglong, _P, _P]),
    "echo_selftest_recip1": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_ulonglong, _P, _P]),
    "echo_selftest_scale2": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_ulonglong, _P, _P]),
    "echo_selftest_mp5_accept": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_ulonglong, _P, _P]),
    "echo_selftest_dfma_blocks": (ctypes.c_int, []),
    "echo_selftest_dfma": (ctypes.c_int, [ctypes.c_longlong, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "echo_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)]),
    "echo_batch_workspace_bytes": (ctypes.c_size_t, [_P]),
    "echo_batch_bind": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "echo_batch_config": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "echo_batch_max_blocks_per_sm": (ctypes.c_int, [_P]),
    "echo_batch_graph": (ctypes.c_int, [_P, ctypes.c_int]),
    "echo_batch_mode": (ctypes.c_int, [_P, ctypes.c_int]),
    "echo_batch_branches": (ctypes.c_int, [_P, ctypes.c_int]),
    "echo_batch_step": (ctypes.c_int, [_P, ctypes.c_double]),
    "echo_batch_last_error": (ctypes.c_char_p, [_P]),
    "echo_batch_destroy": (None, [_P]),
    "echo_mlp_init": (ctypes.c_int, [_P, ctypes.c_ulonglong, _P]),
    "echo_mlp_work_bytes": (ctypes.c_size_t, [ctypes.c_int]),
    "echo_mlp_normalize": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, _P, ctypes.c_size_t, _P]),
    "echo_mlp_train": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_longlong, ctypes.c_float, ctypes.c_double, _P, ctypes.c_size_t,
                                      _P, _P]),
    "echo_mlp_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int,
                                     ctypes.c_double, _P, _P, _P, ctypes.c_size_t, _P]),
    "echo_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P, _P]),
    "echo_mlp_forward_tc": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P, _P]),
    "echo_mlp_guess_error": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, ctypes.c_double, ctypes.c_int, _P, _P,
                                            _P]),
    "echo_mlp_calibrate": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, ctypes.c_double, _P, _P, _P]),
    "echo_mlp_dataset": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong]),
    "echo_mlp_load": (ctypes.c_int, [_P, _P]),
    "echo_set_c2p_guess": (ctypes.c_int, [_P, ctypes.c_int]),
    "echo_totals_static": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                          _P, _P]),
    "echo_last_error": (ctypes.c_char_p, [_P]),
    "echo_destroy": (None, [_P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library.  Raises if it
    cannot be built or loaded -- there is no CPU fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_needed and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(ctx, rc):
    if rc != ECHO_OK:
        msg = load().echo_last_error(ctx) if ctx else b""
        raise EchoError(rc, (msg or b"").decode())


def _ptr(a, writable=False):
    """(pointer, on_device) of a NumPy array (0), a torch CUDA tensor (1) or
    a page-locked torch CPU tensor (2), FP64."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("host arrays must be C-contiguous float64")
        if writable and not a.flags["WRITEABLE"]:
            raise TypeError("output array is read-only")
        return a.ctypes.data, 0
    # torch tensor
    import torch
    if not isinstance(a, torch.Tensor):
        raise TypeError(f"unsupported array type {type(a)}")
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise TypeError("tensors must be contiguous float64")
    if a.is_cuda:
        return a.data_ptr(), 1
    # page-locked host memory is read/written directly by the kernels (2)
    return a.data_ptr(), (2 if a.is_pinned() else 0)


# ---------------------------------------------------------------- entry points

def echo_init(grid: echo_grid, metric: echo_metric, eos: echo_eos, precision: int, cfl: float):
    ctx = _P()
    rc = load().echo_init(ctypes.byref(grid), ctypes.byref(metric), ctypes.byref(eos), int(precision),
                          float(cfl), ctypes.byref(ctx))
    _check(None, rc)
    return ctx


def echo_set_order(ctx, order):
    _check(ctx, load().echo_set_order(ctx, int(order)))


def echo_workspace_bytes(ctx) -> int:
    return int(load().echo_workspace_bytes(ctx))


def echo_state_count(ctx) -> int:
    return int(load().echo_state_count(ctx))


def echo_bind(ctx, dev_ptr: int, nbytes: int, stream_handle: int):
    _check(ctx, load().echo_bind(ctx, _P(dev_ptr), ctypes.c_size_t(nbytes), _P(stream_handle)))


def echo_set_prims(ctx, prims5, bface):
    p, dp = _ptr(prims5)
    f, df = _ptr(bface)
    if dp != df:
        raise TypeError("prims and face field must both be host or both be device arrays")
    _check(ctx, load().echo_set_prims(ctx, _P(p), _P(f), dp))


def echo_set_state(ctx, state, Z=None):
    s, ds = _ptr(state)
    z, dz = _ptr(Z)
    if Z is not None and dz != ds:
        raise TypeError("state and Z must both be host or both be device arrays")
    _check(ctx, load().echo_set_state(ctx, _P(s), _P(z) if z else None, ds))


def echo_get_state(ctx, out):
    p, d = _ptr(out, writable=True)
    _check(ctx, load().echo_get_state(ctx, _P(p), d))
    return out


def echo_get_prims(ctx, out):
    p, d = _ptr(out, writable=True)
    _check(ctx, load().echo_get_prims(ctx, _P(p), d))
    return out


def echo_get_z(ctx, out):
    p, d = _ptr(out, writable=True)
    _check(ctx, load().echo_get_z(ctx, _P(p), d))
    return out


def echo_c2p(ctx, guess_mode: int = 0, stats: echo_totals | None = None):
    rc = load().echo_c2p(ctx, int(guess_mode), ctypes.byref(stats) if stats is not None else None)
    _check(ctx, rc)
    return stats


def echo_rhs(ctx, out):
    p, d = _ptr(out, writable=True)
    _check(ctx, load().echo_rhs(ctx, _P(p), d))
    return out


def echo_step(ctx, dt: float = 0.0):
    _check(ctx, load().echo_step(ctx, float(dt)))


def echo_reduce(ctx) -> echo_totals:
    t = echo_totals()
    _check(ctx, load().echo_reduce(ctx, ctypes.byref(t)))
    return t


ECHO_NK = 14


def echo_profile(ctx, enable: bool):
    _check(ctx, load().echo_profile(ctx, 1 if enable else 0))


def echo_profile_read(ctx) -> dict:
    """{kernel name: (total ms, launches)} since the last read."""
    ms = (ctypes.c_double * ECHO_NK)()
    n = (ctypes.c_longlong * ECHO_NK)()
    _check(ctx, load().echo_profile_read(ctx, ms, n, ECHO_NK))
    return {echo_kernel_name(k): (ms[k], n[k]) for k in range(ECHO_NK)}


def echo_kernel_name(k: int) -> str:
    return (load().echo_kernel_name(int(k)) or b"").decode()


def static_state_count(n) -> int:
    """Doubles of a host-layout state of an n[0] x n[1] x n[2] grid (the
    length echo_totals_static reads)."""
    nx, ny, nz = (int(v) for v in n)
    return 5 * nx * ny * nz + nz * ny * (nx + 1) + nz * (ny + 1) * nx + (nz + 1) * ny * nx


def echo_totals_static(state, n, dx, out6, stream_handle: int = 0):
    """Totals of a device state (torch CUDA tensor, FP64 host layout) into
    the device tensor out6 (6 doubles), allocating nothing.  For callers
    that cannot allocate device memory; see include/echo.h.

    The C entry point cannot see the tensors' lengths or devices, so they
    are checked here before anything is called: a state shorter than the
    grid's host layout, an out6 of fewer than 6 doubles, or a tensor on
    another device than the current one raise ValueError."""
    if len(n) != 3 or len(dx) != 3 or any(int(v) < 1 for v in n):
        raise ValueError("n and dx need 3 entries, n >= 1")
    need = static_state_count(n)
    if state.numel() < need:
        raise ValueError(f"state holds {state.numel()} doubles, the {tuple(n)} grid needs {need}")
    if out6.numel() < 6:
        raise ValueError(f"out6 holds {out6.numel()} doubles, needs 6")
    s, ds = _ptr(state)
    o, do = _ptr(out6, writable=True)
    if not (ds == 1 and do == 1):
        raise TypeError("echo_totals_static takes device arrays")
    import torch
    cur = torch.cuda.current_device()
    if state.device.index != cur or out6.device.index != cur:
        raise ValueError(f"state and out6 must be on the current device cuda:{cur}")
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    dd = (ctypes.c_double * 3)(*[float(v) for v in dx])
    rc = load().echo_totals_static(_P(s), nn, dd, _P(o), _P(stream_handle))
    if rc != ECHO_OK:
        raise EchoError(rc, "echo_totals_static")
    return out6


# ---------------------------------------------------------------- c2p-guess network

ECHO_MLP_NPARAM = 4995
ECHO_MLP_BLOCK = 5024
ECHO_MLP_STATE = 3 * ECHO_MLP_BLOCK


def _dev_f32(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return t.data_ptr()


def _dev_any(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA tensor")
    return t.data_ptr()


def _plain(rc, what):
    if rc != ECHO_OK:
        raise EchoError(rc, what)


def echo_mlp_init(state, seed: int, stream_handle: int = 0):
    _plain(load().echo_mlp_init(_P(_dev_f32(state, "state")), ctypes.c_ulonglong(seed), _P(stream_handle)),
           "echo_mlp_init")


def echo_mlp_work_bytes(batch: int) -> int:
    return int(load().echo_mlp_work_bytes(int(batch)))


def echo_mlp_normalize(state, X, Y, n, work, stream_handle: int = 0):
    _plain(load().echo_mlp_normalize(_P(_dev_f32(state, "state")), _P(_dev_f32(X, "X")), _P(_dev_f32(Y, "Y")),
                                     int(n), _P(_dev_any(work, "work")), work.numel() * work.element_size(),
                                     _P(stream_handle)), "echo_mlp_normalize")


def echo_mlp_train(state, X, Y, n, batch, nsteps, step0, lr, gamma, work, losses=None, stream_handle: int = 0):
    lp = _P(_dev_f32(losses, "losses")) if losses is not None else None
    _plain(load().echo_mlp_train(_P(_dev_f32(state, "state")), _P(_dev_f32(X, "X")), _P(_dev_f32(Y, "Y")),
                                 int(n), int(batch), int(nsteps), int(step0), float(lr), float(gamma),
                                 _P(_dev_any(work, "work")), work.numel() * work.element_size(), lp,
                                 _P(stream_handle)), "echo_mlp_train")


def echo_mlp_grad(state, X, Y, n, row0, batch, gamma, grad, loss, work, stream_handle: int = 0):
    _plain(load().echo_mlp_grad(_P(_dev_f32(state, "state")), _P(_dev_f32(X, "X")), _P(_dev_f32(Y, "Y")),
                                int(n), int(row0), int(batch), float(gamma), _P(_dev_f32(grad, "grad")),
                                _P(_dev_f32(loss, "loss")) if loss is not None else None,
                                _P(_dev_any(work, "work")), work.numel() * work.element_size(),
                                _P(stream_handle)), "echo_mlp_grad")


def echo_mlp_forward(state, X, n, out, stream_handle: int = 0):
    _plain(load().echo_mlp_forward(_P(_dev_f32(state, "state")), _P(_dev_f32(X, "X")), int(n),
                                   _P(_dev_f32(out, "out")), _P(stream_handle)), "echo_mlp_forward")


def echo_mlp_forward_tc(state, X, n, out, stream_handle: int = 0):
    _plain(load().echo_mlp_forward_tc(_P(_dev_f32(state, "state")), _P(_dev_f32(X, "X")), int(n),
                                      _P(_dev_f32(out, "out")), _P(stream_handle)), "echo_mlp_forward_tc")


def echo_mlp_guess_error(state, X, Y, n, gamma, tensor_cores, out, err, stream_handle: int = 0):
    _plain(load().echo_mlp_guess_error(_P(_dev_f32(state, "state")), _P(_dev_f32(X, "X")), _P(_dev_f32(Y, "Y")),
                                       int(n), float(gamma), 1 if tensor_cores else 0, _P(_dev_f32(out, "out")),
                                       _P(_dev_f32(err, "err")), _P(stream_handle)), "echo_mlp_guess_error")


ECHO_MLP_GATE = 5019


def echo_mlp_calibrate(state, X, Y, n, gamma, out, err, stream_handle: int = 0):
    _plain(load().echo_mlp_calibrate(_P(_dev_f32(state, "state")), _P(_dev_f32(X, "X")), _P(_dev_f32(Y, "Y")),
                                     int(n), float(gamma), _P(_dev_f32(out, "out")), _P(_dev_f32(err, "err")),
                                     _P(stream_handle)), "echo_mlp_calibrate")


def echo_mlp_dataset(ctx, X, Y, capacity, offset, stride):
    _check(ctx, load().echo_mlp_dataset(ctx, _P(_dev_f32(X, "X")), _P(_dev_f32(Y, "Y")), int(capacity),
                                        int(offset), int(stride)))


def echo_mlp_load(ctx, state):
    _check(ctx, load().echo_mlp_load(ctx, _P(_dev_f32(state, "state"))))


def echo_set_c2p_guess(ctx, mode: int):
    _check(ctx, load().echo_set_c2p_guess(ctx, int(mode)))


def echo_counters(ctx) -> echo_totals:
    t = echo_totals()
    _check(ctx, load().echo_counters(ctx, ctypes.byref(t)))
    return t


# ---------------------------------------------------------------- batches

def _bcheck(b, rc):
    if rc != ECHO_OK:
        msg = load().echo_batch_last_error(b) if b else b""
        raise EchoError(rc, (msg or b"").decode())


def echo_batch_create(ctxs):
    arr = (_P * len(ctxs))(*[c.value if isinstance(c, _P) else c for c in ctxs])
    b = _P()
    _bcheck(None, load().echo_batch_create(arr, len(ctxs), ctypes.byref(b)))
    return b


def echo_batch_workspace_bytes(b) -> int:
    return int(load().echo_batch_workspace_bytes(b))


def echo_batch_bind(b, dev_ptr, nbytes, stream_handle):
    _bcheck(b, load().echo_batch_bind(b, _P(dev_ptr), ctypes.c_size_t(nbytes), _P(stream_handle)))


def echo_batch_config(b, tile, blocks_per_sm, dynamic_queue):
    _bcheck(b, load().echo_batch_config(b, int(tile), int(blocks_per_sm), int(dynamic_queue)))


def echo_batch_max_blocks_per_sm(b) -> int:
    return int(load().echo_batch_max_blocks_per_sm(b))


def echo_batch_mode(b, mode):
    _bcheck(b, load().echo_batch_mode(b, int(mode)))


def echo_batch_branches(b, branches):
    _bcheck(b, load().echo_batch_branches(b, int(branches)))


def echo_batch_graph(b, enable):
    _bcheck(b, load().echo_batch_graph(b, 1 if enable else 0))


def echo_batch_step(b, dt=0.0):
    _bcheck(b, load().echo_batch_step(b, float(dt)))


def echo_batch_destroy(b):
    load().echo_batch_destroy(b)


def echo_selftest_dfma_blocks() -> int:
    return int(load().echo_selftest_dfma_blocks())


def echo_selftest_dfma(iters, dev_out, stream_handle: int = 0) -> float:
    """Launch the FP64 FMA throughput probe; returns the launch's flop count.
    dev_out: a device tensor of at least 256 * echo_selftest_dfma_blocks()
    doubles."""
    need = 256 * echo_selftest_dfma_blocks()
    if dev_out.numel() < need or dev_out.element_size() != 8:
        raise ValueError(f"dev_out needs {need} doubles")
    f = ctypes.c_double(0.0)
    _plain(load().echo_selftest_dfma(int(iters), _P(_dev_any(dev_out, "out")), ctypes.byref(f), _P(stream_handle)),
           "echo_selftest_dfma")
    return f.value


def echo_selftest_scale2(n, seed, dev_mismatch, stream_handle: int = 0):
    _plain(load().echo_selftest_scale2(int(n), ctypes.c_ulonglong(seed), _P(_dev_any(dev_mismatch, "mismatch")),
                                       _P(stream_handle)), "echo_selftest_scale2")


def echo_selftest_mp5_accept(n, seed, dev_mismatch, stream_handle: int = 0):
    _plain(load().echo_selftest_mp5_accept(int(n), ctypes.c_ulonglong(seed), _P(_dev_any(dev_mismatch, "mismatch")),
                                           _P(stream_handle)), "echo_selftest_mp5_accept")


def echo_selftest_recip(n, seed, dev_max, stream_handle: int = 0):
    _plain(load().echo_selftest_recip(int(n), ctypes.c_ulonglong(seed), _P(_dev_any(dev_max, "max")),
                                      _P(stream_handle)), "echo_selftest_recip")


def echo_selftest_recip1(n, seed, dev_max, stream_handle: int = 0):
    _plain(load().echo_selftest_recip1(int(n), ctypes.c_ulonglong(seed), _P(_dev_any(dev_max, "max")),
                                       _P(stream_handle)), "echo_selftest_recip1")


def echo_selftest_conversions(n, seed, dev_counter, stream_handle: int = 0):
    _plain(load().echo_selftest_conversions(int(n), ctypes.c_ulonglong(seed), _P(_dev_any(dev_counter, "counter")),
                                            _P(stream_handle)), "echo_selftest_conversions")


def echo_last_error(ctx) -> str:
    return (load().echo_last_error(ctx) or b"").decode()


def echo_destroy(ctx):
    load().echo_destroy(ctx)
