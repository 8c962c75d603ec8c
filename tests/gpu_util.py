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


def l1_frame(orc, prob, g, o):
    """Relative L1 errors of a state g against o that stay well conditioned
    for vector components near zero: D and tau as sum|g - o| / sum|o|;
    each covariant momentum component S_i in the local orthonormal frame,
    sum |dS_i| sqrt(gamma^ii) / sum |S| with |S| = sqrt(gamma^ij S_i S_j);
    each field component likewise from the cell-centre B~ (mean of the two
    faces), sum |dB^i| sqrt(gamma_ii) / sum |B| with |B| = sqrt(gamma_ij B^i
    B^j).  Metric from the oracle's closed form at the cell centres (it
    depends on x1 and x2 only)."""
    cfg = orc.make_cfg(prob)
    nx, ny, nz = prob.n
    gi = np.zeros((3, 3, ny, nx))
    gl = np.zeros((3, 3, ny, nx))
    for j in range(ny):
        for i in range(nx):
            m = orc.metric_point(cfg, [prob.x0[0] + (i + 0.5) * prob.dx[0], prob.x0[1] + (j + 0.5) * prob.dx[1],
                                       prob.x0[2] + 0.5 * prob.dx[2]])
            gi[:, :, j, i] = m["gi"]
            gl[:, :, j, i] = m["g"]

    def centre(st):
        cells, bx, by, bz = orc.split_state(st, prob.n)
        B = np.stack([0.5 * (bx[:, :, :-1] + bx[:, :, 1:]), 0.5 * (by[:, :-1, :] + by[:, 1:, :]),
                      0.5 * (bz[:-1] + bz[1:])])
        return cells, B

    cg, Bg = centre(g)
    co, Bo = centre(o)
    out = {"D": l1_rel(cg[0], co[0]), "tau": l1_rel(cg[4], co[4])}
    S = co[1:4]
    Smag = np.sqrt(np.einsum("ijyx,izyx,jzyx->zyx", gi, S, S))
    for q in range(3):
        out[f"S_{q + 1}"] = float(np.sum(np.abs(cg[1 + q] - co[1 + q]) * np.sqrt(gi[q, q])) / np.sum(Smag))
    Bmag = np.sqrt(np.einsum("ijyx,izyx,jzyx->zyx", gl, Bo, Bo))
    for q in range(3):
        out[f"B_{q + 1}"] = float(np.sum(np.abs(Bg[q] - Bo[q]) * np.sqrt(gl[q, q])) / np.sum(Bmag))
    return out
