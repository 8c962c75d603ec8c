"""Helpers shared by the GPU tests: run a problem on the GPU through the
C-ABI binding and on the oracle, and compare field by field."""
import numpy as np

FIELDS = ["D", "S_x", "S_y", "S_z", "tau", "Bx", "By", "Bz"]


def fields(orc, state, n):
    cells, bx, by, bz = orc.split_state(state, n)
    return [cells[0], cells[1], cells[2], cells[3], cells[4], bx, by, bz]


def max_rel(g, o):
    """max |g - o| / max |o| (a pointwise relative error is undefined for
    fields that cross zero)."""
    den = np.max(np.abs(o))
    if den == 0.0:
        return float(np.max(np.abs(g)))
    return float(np.max(np.abs(g - o)) / den)


def l1_rel(g, o):
    den = np.sum(np.abs(o))
    return float(np.sum(np.abs(g - o)) / den) if den > 0 else float(np.sum(np.abs(g)))


def per_field(orc, gs, os_, n, metric=max_rel):
    return {name: metric(a, b) for name, a, b in zip(FIELDS, fields(orc, gs, n), fields(orc, os_, n))}


def gpu_run(prob, nsteps, precision=64, dt=0.0):
    from paper_1810_04597_gb300.echo import Solver
    s = Solver(prob, precision=precision)
    s.set_prims()
    for _ in range(nsteps):
        s.step(dt)
    return s.get_state(), s


def oracle_run(orc, prob, nsteps, dt=0.0):
    cfg = orc.make_cfg(prob)
    st, Z = orc.p2c(cfg, prob.prims, prob.bface)
    if nsteps == 0:
        return st, Z, np.zeros(0), None
    return orc.steps(cfg, st, Z, nsteps, dt)
