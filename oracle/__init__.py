"""Plain FP64 CPU oracle of the per-step GRMHD update (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never does, and this package never imports the library.

The arithmetic lives in ``echo_oracle.c`` (plain C, FP64, built with
``-O2 -ffp-contract=off``); this module only compiles it and marshals NumPy
arrays.  Every function says which step of the scheme it exposes; the C
source cites the published method each step restates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "echo_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "mlp_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libecho_oracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, OUTFLOW, AXIS = 0, 1, 2


class OCfg(ctypes.Structure):
    """Mirror of the oracle's ``ocfg`` struct."""

    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("x0", ctypes.c_double * 3),
        ("dx", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 6),
        ("metric", ctypes.c_int),
        ("spin", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("floors", ctypes.c_int),
        ("rho_floor", ctypes.c_double),
        ("rho_floor_pow", ctypes.c_double),
        ("p_floor", ctypes.c_double),
        ("p_floor_pow", ctypes.c_double),
        ("order", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libecho_oracle.so``."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        if (not force and os.path.exists(_LIB)
                and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-fopenmp", "-std=c11", "-Wall", "-Wno-unused-variable", "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _LIB)
        return _LIB


_COUNT_SRC = os.path.join(_HERE, "op_count.cpp")
_COUNT_LIB = os.path.join(_BUILD, "libecho_oracle_count.so")
_count_lib = None
COUNT_PHASES = ("c2p", "cfl", "faces", "emf", "correct", "assemble", "ct", "rk", "other")
COUNT_OPS = ("add", "mul", "div", "sqrt", "fn")


def build_count(force: bool = False) -> str:
    """Compile the operation-counting build (op_count.cpp: echo_oracle.c as
    C++ with a counting number type, OpenMP as the plain build) into
    ``oracle/_build/libecho_oracle_count.so``."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        if (not force and os.path.exists(_COUNT_LIB)
                and all(os.path.getmtime(_COUNT_LIB) >= os.path.getmtime(f) for f in (_SRC, _COUNT_SRC))):
            return _COUNT_LIB
        tmp = _COUNT_LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c++17", "-fopenmp",
               "-Wall", "-Wno-unused-variable", "-o", tmp, _COUNT_SRC]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _COUNT_LIB)
        return _COUNT_LIB


def count_lib():
    """The counting build, with the entry points the counts need."""
    global _count_lib
    if _count_lib is None:
        L = ctypes.CDLL(build_count())
        P = ctypes.POINTER
        d, i, ll = ctypes.c_double, ctypes.c_int, ctypes.c_longlong
        pc, pd = P(OCfg), P(d)
        L.oracle_p2c.argtypes = [pc, pd, pd, pd, pd]
        L.oracle_p2c.restype = i
        L.oracle_steps.argtypes = [pc, pd, pd, i, d, pd, P(ll)]
        L.oracle_steps.restype = i
        L.oracle_c2p.argtypes = [pc, pd, pd, pd, pd, P(ll)]
        L.oracle_c2p.restype = i
        L.oracle_mp5_face.argtypes = [pd]
        L.oracle_mp5_face.restype = d
        L.oracle_count_reset.argtypes = [i, i]
        L.oracle_count_read.argtypes = [P(ll), P(ll), P(ll)]
        L.oracle_count_nphase.restype = i
        _count_lib = L
    return _count_lib


def count_read() -> dict:
    """Counts since the last count_reset: {phase: {op: n, ..., "flops",
    "units", "sampled", "per_unit"}} (per_unit: flops over the sampled
    units)."""
    L = count_lib()
    nph = L.oracle_count_nphase()
    c = (ctypes.c_longlong * (nph * len(COUNT_OPS)))()
    u = (ctypes.c_longlong * nph)()
    sm = (ctypes.c_longlong * nph)()
    L.oracle_count_read(c, u, sm)
    out = {}
    for p in range(nph):
        row = {op: int(c[p * len(COUNT_OPS) + k]) for k, op in enumerate(COUNT_OPS)}
        row["flops"] = row["add"] + row["mul"] + row["div"] + row["sqrt"]
        row["units"] = int(u[p])
        row["sampled"] = int(sm[p])
        row["per_unit"] = row["flops"] / row["sampled"] if sm[p] else None
        out[COUNT_PHASES[p]] = row
    return out


def count_reset(sample_every: int = 1, cse: bool = False):
    count_lib().oracle_count_reset(int(sample_every), 1 if cse else 0)


def count_mp5_face(u5, cse: bool = False) -> tuple:
    """(value, counts) of one MP5 interface value in the counting build:
    the operations of a single reconstruction (outside any step)."""
    count_reset(1, cse)
    v = count_lib().oracle_mp5_face(_dp(_f64(u5)))
    return v, count_read()["other"]


def count_steps(cfg: OCfg, prims5: np.ndarray, bface: np.ndarray, nsteps: int, dt: float = 0.0,
                sample_every: int = 1, cse: bool = False, state=None, Z=None):
    """Operation counts of nsteps SSP-RK3 steps of the counting build, from
    the primitives (the initial p2c is not counted) or, if given, from the
    conserved state and Newton memory (state, Z); returns (counts per phase
    as count_read gives them, c2p stats: iterations, calls, fails, floors,
    fallback faces)."""
    L = count_lib()
    n = list(cfg.n)
    N = n[0] * n[1] * n[2]
    if state is None:
        state = np.zeros(state_count(n))
        Z = np.zeros(N)
        count_reset(1, False)
        _check(L.oracle_p2c(ctypes.byref(cfg), _dp(_f64(prims5)), _dp(_f64(bface)), _dp(state), _dp(Z)), "p2c")
    else:
        state = _f64(state).copy()
        Z = _f64(Z).copy()
    count_reset(sample_every, cse)
    dts = np.zeros(max(int(nsteps), 1))
    stats = (ctypes.c_longlong * 6)()
    _check(L.oracle_steps(ctypes.byref(cfg), _dp(state), _dp(Z), int(nsteps), float(dt), _dp(dts), stats),
           "steps")
    return count_read(), dict(iters=stats[0], calls=stats[1], fails=stats[2], floors=stats[3],
                              fallback_faces=stats[4], guard_faces=stats[5])


def lib():
    global _lib
    if _lib is None:
        # ECHO_ORACLE_LIB: a prebuilt variant of the oracle (the planted-mistake
        # tests load deliberately broken copies this way)
        path = os.environ.get("ECHO_ORACLE_LIB") or build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i, ll = ctypes.c_double, ctypes.c_int, ctypes.c_longlong
        pc = P(OCfg)
        pd = P(d)
        L.oracle_metric_point.argtypes = [pc, pd, pd]
        L.oracle_p2c_point.argtypes = [pc, pd, pd, pd]
        L.oracle_c2p_point.argtypes = [pc, pd, pd, pd, d, pd, pd, P(i)]
        L.oracle_c2p_point.restype = i
        L.oracle_c2p_residual.argtypes = [pc, pd, pd, pd, d, pd, pd]
        L.oracle_mp5_face.argtypes = [pd]
        L.oracle_mp5_face.restype = d
        L.oracle_mp5_unlimited.argtypes = [pd]
        L.oracle_mp5_unlimited.restype = d
        L.oracle_mp5_face_order.argtypes = [pd, i]
        L.oracle_mp5_face_order.restype = d
        L.oracle_ho_flux.argtypes = [pd]
        L.oracle_ho_flux.restype = d
        L.oracle_ho_center.argtypes = [pd]
        L.oracle_ho_center.restype = d
        L.oracle_ghosts.restype = i
        L.oracle_set_threads.argtypes = [i]
        L.oracle_get_threads.restype = i
        L.oracle_fill_padded.argtypes = [pc, pd, i, i, i]
        L.oracle_speeds_point.argtypes = [pc, pd, pd, i, pd, pd]
        L.oracle_flux_point.argtypes = [pc, pd, pd, i, pd, pd]
        L.oracle_hll.argtypes = [pd, pd, pd, pd, d, d, pd]
        L.oracle_sources_point.argtypes = [pc, pd, pd, pd]
        L.oracle_state_count.argtypes = [P(i)]
        L.oracle_state_count.restype = ctypes.c_size_t
        L.oracle_p2c.argtypes = [pc, pd, pd, pd, pd]
        L.oracle_p2c.restype = i
        L.oracle_c2p.argtypes = [pc, pd, pd, pd, pd, P(ll)]
        L.oracle_c2p.restype = i
        L.oracle_rhs.argtypes = [pc, pd, pd, pd, pd]
        L.oracle_rhs.restype = i
        L.oracle_steps.argtypes = [pc, pd, pd, i, d, pd, P(ll)]
        L.oracle_steps.restype = i
        L.oracle_reduce.argtypes = [pc, pd, pd]
        L.oracle_reduce.restype = i
        L.oracle_mlp_nparam.restype = i
        L.oracle_mlp_forward.argtypes = [pd, pd, i, pd]
        L.oracle_mlp_targets.argtypes = [pd, pd, pd, i, d, pd]
        L.oracle_mlp_loss_grad.argtypes = [pd, pd, pd, i, d, d, pd, pd]
        L.oracle_mlp_loss_grad.restype = d
        L.oracle_mlp_adam.argtypes = [pd, pd, pd, pd, i, d, d, d, d]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_cfg(problem) -> OCfg:
    """Build the oracle config from a problem description (any object with
    the attributes of ``paper_1810_04597_gb300.inputs.Problem``)."""
    c = OCfg()
    for d in range(3):
        c.n[d] = int(problem.n[d])
        c.x0[d] = float(problem.x0[d])
        c.dx[d] = float(problem.dx[d])
    for s in range(6):
        c.bc[s] = int(problem.bc[s])
    c.metric = int(problem.metric)
    c.spin = float(problem.spin)
    c.gamma = float(problem.gamma)
    c.cfl = float(problem.cfl)
    c.floors = int(bool(problem.floors))
    c.rho_floor = float(problem.rho_floor)
    c.rho_floor_pow = float(problem.rho_floor_pow)
    c.p_floor = float(problem.p_floor)
    c.p_floor_pow = float(problem.p_floor_pow)
    c.order = int(getattr(problem, "order", 0))
    return c


def state_count(n) -> int:
    arr = (ctypes.c_int * 3)(*[int(v) for v in n])
    return int(lib().oracle_state_count(arr))


# ---------------------------------------------------------------- pointwise

def metric_point(cfg: OCfg, x):
    """alpha, beta^i, gamma_ij, gamma^ij, sqrt(gamma) at coordinate x."""
    out = np.zeros(23)
    lib().oracle_metric_point(ctypes.byref(cfg), _dp(_f64(x)), _dp(out))
    return dict(alpha=out[0], beta=out[1:4].copy(), g=out[4:13].reshape(3, 3).copy(),
                gi=out[13:22].reshape(3, 3).copy(), sqrtg=out[22])


def p2c_point(cfg: OCfg, x, P8):
    """Undensitised (D, S_j, tau) of primitives (rho, v^i, p, B^i)."""
    out = np.zeros(5)
    lib().oracle_p2c_point(ctypes.byref(cfg), _dp(_f64(x)), _dp(_f64(P8)), _dp(out))
    return out


def c2p_point(cfg: OCfg, x, C5, B3, Zguess):
    """Newton c2p at one point: (status, P5, Z, iterations)."""
    P5 = np.zeros(5)
    Z = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    rc = lib().oracle_c2p_point(ctypes.byref(cfg), _dp(_f64(x)), _dp(_f64(C5)), _dp(_f64(B3)),
                                float(Zguess), _dp(P5), ctypes.byref(Z), ctypes.byref(it))
    return rc, P5, Z.value, it.value


def c2p_residual(cfg: OCfg, x, C5, B3, Z):
    f = ctypes.c_double(0.0)
    fp = ctypes.c_double(0.0)
    lib().oracle_c2p_residual(ctypes.byref(cfg), _dp(_f64(x)), _dp(_f64(C5)), _dp(_f64(B3)),
                              float(Z), ctypes.byref(f), ctypes.byref(fp))
    return f.value, fp.value


def mp5_face(u5) -> float:
    return lib().oracle_mp5_face(_dp(_f64(u5)))


def mp5_face_order(u5, order):
    """MP5 interface value with the cell-average (order 0) or point-value
    (order 1) interpolant."""
    return lib().oracle_mp5_face_order(_dp(_f64(u5)), int(order))


def ho_flux(f5):
    """Flux-derivative correction F - D2/24 + 3 D4/640 at the middle of five
    interface values."""
    return lib().oracle_ho_flux(_dp(_f64(f5)))


def ho_center(b6):
    """Sixth-order midpoint interpolation of six equally spaced values."""
    return lib().oracle_ho_center(_dp(_f64(b6)))


def set_threads(n: int):
    """Threads of the oracle's OpenMP loops from now on."""
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def ghosts() -> int:
    """Ghost layers per side of the oracle's padded arrays."""
    return int(lib().oracle_ghosts())


def fill_padded(cfg: OCfg, a: np.ndarray, comp: int, face: int, dens: int = 0) -> np.ndarray:
    """The oracle's ghost fill applied to a copy of a padded array of shape
    (n2 + 2g, n1 + 2g, n0 + 2g); comp = the vector component it holds (-1
    for a scalar), face = its face direction (-1 for a cell array), dens = 1
    for an array carrying the factor sqrt(gamma) (the densitised face
    field), which is odd about a polar axis."""
    g = ghosts()
    shape = tuple(cfg.n[2 - k] + 2 * g for k in range(3))
    out = _f64(a).copy()
    assert out.shape == shape, (out.shape, shape)
    lib().oracle_fill_padded(ctypes.byref(cfg), _dp(out), int(comp), int(face), int(dens))
    return out


def mp5_unlimited(u5) -> float:
    return lib().oracle_mp5_unlimited(_dp(_f64(u5)))


def speeds_point(cfg: OCfg, x, P8, d):
    lp = ctypes.c_double(0.0)
    lm = ctypes.c_double(0.0)
    lib().oracle_speeds_point(ctypes.byref(cfg), _dp(_f64(x)), _dp(_f64(P8)), int(d),
                              ctypes.byref(lp), ctypes.byref(lm))
    return lp.value, lm.value


def flux_point(cfg: OCfg, x, P8, d):
    """(F, U) along d, both times sqrt(gamma)."""
    F = np.zeros(5)
    U = np.zeros(5)
    lib().oracle_flux_point(ctypes.byref(cfg), _dp(_f64(x)), _dp(_f64(P8)), int(d), _dp(F), _dp(U))
    return F, U


def hll(FL, FR, UL, UR, ap, am):
    F = np.zeros(5)
    lib().oracle_hll(_dp(_f64(FL)), _dp(_f64(FR)), _dp(_f64(UL)), _dp(_f64(UR)), float(ap), float(am),
                     _dp(F))
    return F


def sources_point(cfg: OCfg, x, P8):
    out = np.zeros(5)
    lib().oracle_sources_point(ctypes.byref(cfg), _dp(_f64(x)), _dp(_f64(P8)), _dp(out))
    return out


# ---------------------------------------------------------------- grid level

def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def p2c(cfg: OCfg, prims5: np.ndarray, bface: np.ndarray):
    """Primitives (5, nz, ny, nx) and face field (host face layout, flat) ->
    (state in host layout, Z)."""
    n = list(cfg.n)
    N = n[0] * n[1] * n[2]
    prims5 = _f64(prims5).reshape(-1)
    bface = _f64(bface).reshape(-1)
    state = np.zeros(state_count(n))
    Z = np.zeros(N)
    _check(lib().oracle_p2c(ctypes.byref(cfg), _dp(prims5), _dp(bface), _dp(state), _dp(Z)), "p2c")
    return state, Z


def c2p(cfg: OCfg, state: np.ndarray, Zguess: np.ndarray | None = None, check: bool = True):
    """c2p of a state -> (prims8 (8, N), Z, stats dict, status)."""
    n = list(cfg.n)
    N = n[0] * n[1] * n[2]
    state = _f64(state)
    prims = np.zeros(8 * N)
    Z = np.zeros(N)
    stats = (ctypes.c_longlong * 4)()
    zg = _f64(Zguess) if Zguess is not None else np.zeros(N)
    rc = lib().oracle_c2p(ctypes.byref(cfg), _dp(state), _dp(zg), _dp(prims), _dp(Z), stats)
    if check:
        _check(rc, "c2p")
    return prims.reshape(8, N), Z, dict(iters=stats[0], calls=stats[1], fails=stats[2],
                                        floors=stats[3]), rc


def rhs(cfg: OCfg, state: np.ndarray, Z: np.ndarray):
    """L(U) in host layout; returns (L, Z_after, rate_max)."""
    state = _f64(state)
    Z = _f64(Z).copy()
    L = np.zeros_like(state)
    rate = ctypes.c_double(0.0)
    _check(lib().oracle_rhs(ctypes.byref(cfg), _dp(state), _dp(Z), _dp(L), ctypes.byref(rate)), "rhs")
    return L, Z, rate.value


def steps(cfg: OCfg, state: np.ndarray, Z: np.ndarray, nsteps: int, dt: float = 0.0):
    """nsteps SSP-RK3 steps; dt <= 0 selects the CFL dt.  Returns
    (state, Z, dts, stats dict: c2p iterations, calls, fails, floors,
    first-order face fallbacks, faces the order-1 safeguard replaced)."""
    state = _f64(state).copy()
    Z = _f64(Z).copy()
    dts = np.zeros(max(int(nsteps), 1))
    stats = (ctypes.c_longlong * 6)()
    rc = lib().oracle_steps(ctypes.byref(cfg), _dp(state), _dp(Z), int(nsteps), float(dt), _dp(dts),
                            stats)
    _check(rc, "steps")
    return state, Z, dts[:nsteps], dict(iters=stats[0], calls=stats[1], fails=stats[2],
                                        floors=stats[3], fallback_faces=stats[4], guard_faces=stats[5])


def reduce(cfg: OCfg, state: np.ndarray):
    """(mass, energy(tau), S_x, S_y, S_z, max|div B~|)."""
    out = np.zeros(6)
    _check(lib().oracle_reduce(ctypes.byref(cfg), _dp(_f64(state)), _dp(out)), "reduce")
    return out


def split_state(state: np.ndarray, n):
    """View a host-layout state as (cells (5, nz, ny, nx), Bx, By, Bz)."""
    nx, ny, nz = (int(v) for v in n)
    N = nx * ny * nz
    cells = state[:5 * N].reshape(5, nz, ny, nx)
    o = 5 * N
    bx = state[o:o + nz * ny * (nx + 1)].reshape(nz, ny, nx + 1)
    o += nz * ny * (nx + 1)
    by = state[o:o + nz * (ny + 1) * nx].reshape(nz, ny + 1, nx)
    o += nz * (ny + 1) * nx
    bz = state[o:o + (nz + 1) * ny * nx].reshape(nz + 1, ny, nx)
    return cells, bx, by, bz


# ---------------------------------------------------------------- c2p-guess network

MLP_NPARAM = 4995
MLP_NNORM = 24


def mlp_forward(params, x):
    """Raw outputs (n, 3) of the network; params = parameters + norm block."""
    params = _f64(params)
    x = _f64(x).reshape(-1, 9)
    out = np.zeros((x.shape[0], 3))
    lib().oracle_mlp_forward(_dp(params), _dp(x), x.shape[0], _dp(out))
    return out


def mlp_targets(params, x, y, gamma=4.0 / 3.0):
    params = _f64(params)
    x = _f64(x).reshape(-1, 9)
    y = _f64(y).reshape(-1, 3)
    t = np.zeros_like(y)
    lib().oracle_mlp_targets(_dp(params), _dp(x), _dp(y), x.shape[0], float(gamma), _dp(t))
    return t


def mlp_loss_grad(params, x, y, gamma=4.0 / 3.0, w2=0.1, t_fixed=None):
    """(mean loss, gradient over the 4995 parameters)."""
    params = _f64(params)
    x = _f64(x).reshape(-1, 9)
    y = _f64(y).reshape(-1, 3)
    g = np.zeros(MLP_NPARAM)
    tf = _dp(_f64(t_fixed)) if t_fixed is not None else None
    loss = lib().oracle_mlp_loss_grad(_dp(params), _dp(x), _dp(y), x.shape[0], float(gamma), float(w2),
                                      _dp(g), tf)
    return loss, g


def mlp_adam(params, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays."""
    lib().oracle_mlp_adam(_dp(params), _dp(m), _dp(v), _dp(_f64(g)), int(t), float(lr), float(b1),
                          float(b2), float(eps))
