"""Kerr-Schild torus on the GPU (metric tables, sources, floors, outflow and
polar-axis boundaries) against the oracle, through the C ABI."""
import numpy as np
import pytest

from paper_1810_04597_gb300 import inputs
from gpu_util import FIELDS, fields, gpu_run, l1_frame, l1_rel, max_rel, oracle_run, per_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def test_ks_p2c_and_c2p(orc):
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.fm_torus((48, 24, 8))
    s = Solver(prob)
    s.set_prims()
    st_g = s.get_state()
    cfg = orc.make_cfg(prob)
    st_o, Z_o = orc.p2c(cfg, prob.prims, prob.bface)
    errs = per_field(orc, st_g, st_o, prob.n)
    assert max(errs.values()) <= 1e-13, errs
    stats = s.c2p(guess_mode=2)
    P_g = s.get_prims()
    P_o, _, ostats, _ = orc.c2p(cfg, st_o, None)
    # velocity and field components are compared against the largest
    # component (v^theta, B^phi vanish in the initial torus)
    vs = np.max(np.abs(P_o[1:4]))
    bs = np.max(np.abs(P_o[5:8]))
    for q in range(8):
        den = vs if 1 <= q <= 3 else (bs if q >= 5 else np.max(np.abs(P_o[q])))
        assert np.max(np.abs(P_g[q] - P_o[q])) <= 1e-12 * den, q
    assert stats["floor_hits"] == ostats["floors"]


def test_ks_rhs_parity(orc):
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.fm_torus((48, 24, 8), seed=5)
    s = Solver(prob)
    s.set_prims()
    L_g = s.rhs()
    cfg = orc.make_cfg(prob)
    st, Z = orc.p2c(cfg, prob.prims, prob.bface)
    L_o, _, _ = orc.rhs(cfg, st, Z)
    errs = per_field(orc, L_g, L_o, prob.n)
    assert max(errs.values()) <= 1e-11, errs


@pytest.mark.parametrize("spin,field", [(0.9, True), (0.0, False)])
def test_ks_ten_step_parity(orc, spin, field):
    prob = inputs.fm_torus((64, 32, 16), spin=spin, with_field=field)
    st_g, s = gpu_run(prob, 10)
    st_o, _, dts, ostats = oracle_run(orc, prob, 10)
    errs = per_field(orc, st_g, st_o, prob.n)
    t = s.reduce()
    diag = dict(errs=errs, gpu=(t["c2p_fail"], t["floor_hits"]), oracle=(ostats["fails"], ostats["floors"]))
    assert max(errs.values()) <= 1e-11, diag
    assert t["c2p_calls"] > 0
    # the polar-axis faces hold B~^theta = 0
    _, _, by, _ = orc.split_state(st_g, prob.n)
    assert np.all(by[:, 0, :] == 0.0) and np.all(by[:, -1, :] == 0.0)


def test_ks_fp32_bulk(orc):
    """FP32 bulk (FP64 c2p, metric and reductions) on the torus against the
    FP64 oracle after 10 steps, at <= 1e-5 relative L1 per field.  S_theta
    and B^phi nearly vanish in the equilibrium, so their plain relative L1
    divides by almost nothing; every vector component is measured in the
    local orthonormal frame against the L1 of the vector's magnitude
    (gpu_util.l1_frame), which is the same number for a component that
    carries the vector and stays well conditioned for one that does not."""
    prob = inputs.fm_torus((64, 32, 16))
    st_g, s = gpu_run(prob, 10, precision=32)
    st_o, _, _, _ = oracle_run(orc, prob, 10)
    plain = per_field(orc, st_g, st_o, prob.n, metric=l1_rel)
    frame = l1_frame(orc, prob, st_g, st_o)
    print("FP32 torus, relative L1 per field:", plain, "frame-normalised:", frame)
    assert max(frame.values()) <= 1e-5, frame


@pytest.mark.parametrize("order", [0, 1])
def test_michel_rhs_parity(orc, order):
    """L(U) of the Michel accretion state (radial inflow through the
    Kerr-Schild shift) on the GPU against the oracle, both orders."""
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.michel_accretion(96, order=order)
    s = Solver(prob)
    s.set_prims()
    L_g = s.rhs()
    cfg = orc.make_cfg(prob)
    st, Z = orc.p2c(cfg, prob.prims, prob.bface)
    L_o, _, _ = orc.rhs(cfg, st, Z)
    errs = per_field(orc, L_g, L_o, prob.n)
    assert max(errs[k] for k in ("D", "S_x", "tau")) <= 1e-11, errs


def test_ks_failed_inversion_takes_the_floor_path(orc):
    """Floors on: an inadmissible cell (tau = -10 D) is not an error; it
    keeps its previous primitives (zero here, nothing inverted before),
    takes the floors and is counted as a failure and a floor hit, exactly as
    the oracle does; every other cell matches the oracle."""
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.fm_torus((48, 24, 8), seed=9)
    cfg = orc.make_cfg(prob)
    st, Z = orc.p2c(cfg, prob.prims, prob.bface)
    N = prob.ncells
    cell = 20 + 48 * (12 + 24 * 3)     # inside the torus, away from the axis
    bad = st.copy()
    bad[4 * N + cell] = -10.0 * bad[cell]
    P_o, _, ostats, rc = orc.c2p(cfg, bad, Z, check=False)
    assert rc == 0 and ostats["fails"] == 1
    s = Solver(prob)
    s.set_state(bad, Z)
    stats = s.c2p(guess_mode=0)
    assert stats["c2p_fail"] == 1
    assert stats["floor_hits"] == ostats["floors"]
    P_g = s.get_prims()
    assert P_g[1:4, cell].tolist() == [0.0, 0.0, 0.0]
    # velocity and field components against their largest component (v^theta
    # vanishes to rounding in the initial torus)
    vs, bs = np.max(np.abs(P_o[1:4])), np.max(np.abs(P_o[5:8]))
    for q in range(8):
        den = vs if 1 <= q <= 3 else (bs if q >= 5 else np.max(np.abs(P_o[q])))
        assert np.max(np.abs(P_g[q] - P_o[q])) <= 1e-12 * den, q


def test_polar_cap_ten_step_parity(orc):
    """A magnetised flow through the polar axis (inputs.polar_cap: B~^r,
    B~^phi odd and B~^theta even about the pole, continued that way into
    the ghosts on both paths) matches the oracle after 10 steps to 1e-11
    per field, and div B~ stays at rounding."""
    prob = inputs.polar_cap((24, 24, 8))
    st_g, s = gpu_run(prob, 10)
    st_o, _, _, _ = oracle_run(orc, prob, 10)
    errs = per_field(orc, st_g, st_o, prob.n)
    assert max(errs.values()) <= 1e-11, errs
    t = s.reduce()
    _, bx, _, _ = orc.split_state(st_g, prob.n)
    assert t["max_divb"] <= 1e-10 * np.max(np.abs(bx)) / min(prob.dx), t["max_divb"]
