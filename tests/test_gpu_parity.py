"""GPU path vs the oracle, element by element, through the C ABI.

Tolerances: FP64 max-relative error per field (normalised by the field's
max-abs) <= 1e-11 after 10 SSP-RK3 steps, the target for the FP64 path;
tighter bounds for single operations, where only rounding order differs.
"""
import numpy as np
import pytest

from paper_1810_04597_gb300 import inputs
from gpu_util import FIELDS, fields, gpu_run, max_rel, oracle_run, per_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1810_04597_gb300 import _lib
    _lib.load()


def test_p2c_parity(orc):
    prob = inputs.smooth_box(32)
    st_g, _ = gpu_run(prob, 0)
    st_o, _, _, _ = oracle_run(orc, prob, 0)
    errs = per_field(orc, st_g, st_o, prob.n)
    assert max(errs.values()) <= 1e-14, errs


def test_c2p_parity(orc):
    """Cold-guess Newton on the GPU vs the oracle's c2p (pointwise)."""
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.sweep_box(24)
    s = Solver(prob)
    s.set_prims()
    stats = s.c2p(guess_mode=2)
    assert stats["c2p_fail"] == 0
    P_g = s.get_prims()
    cfg = orc.make_cfg(prob)
    st_o, Z_o = orc.p2c(cfg, prob.prims, prob.bface)
    P_o, _, ostats, _ = orc.c2p(cfg, st_o, None)
    assert ostats["fails"] == 0
    for q in range(8):
        assert max_rel(P_g[q], P_o[q]) <= 1e-13, q
    # and the input primitives are recovered
    for q in range(5):
        assert max_rel(P_g[q], prob.prims[q].reshape(-1)) <= 1e-13, q
    # the iteration histogram covers every inversion and sums to the
    # iteration count, which matches the oracle's (a cell whose last step
    # lands on the stopping threshold may take one iteration more or less)
    h = np.array(stats["c2p_iter_hist"])
    assert h.sum() == stats["c2p_calls"] == prob.ncells
    assert h[-1] == 0 and int(np.dot(np.arange(h.size), h)) == stats["c2p_iters"]
    assert abs(stats["c2p_iters"] - ostats["iters"]) <= 0.002 * prob.ncells, (stats["c2p_iters"], ostats["iters"])


def test_rhs_parity_ragged(orc):
    """L(U) on a ragged grid (not a multiple of any tile size)."""
    from paper_1810_04597_gb300.echo import Solver
    base = inputs.sweep_box(40, seed=5)
    n = (37, 29, 23)
    prob = crop(base, n)
    s = Solver(prob)
    s.set_prims()
    L_g = s.rhs()
    cfg = orc.make_cfg(prob)
    st, Z = orc.p2c(cfg, prob.prims, prob.bface)
    L_o, _, rate = orc.rhs(cfg, st, Z)
    errs = per_field(orc, L_g, L_o, n)
    assert max(errs.values()) <= 1e-12, errs


def crop(prob, n):
    """A sub-box of a problem's primitives and faces as a new periodic
    problem (the wrap is discontinuous, which is fine: both sides see the
    same data)."""
    nx, ny, nz = n
    prims = np.ascontiguousarray(prob.prims[:, :nz, :ny, :nx])
    N0 = prob.n
    o = 0
    bx = prob.bface[o:o + N0[2] * N0[1] * (N0[0] + 1)].reshape(N0[2], N0[1], N0[0] + 1)
    o += bx.size
    by = prob.bface[o:o + N0[2] * (N0[1] + 1) * N0[0]].reshape(N0[2], N0[1] + 1, N0[0])
    o += by.size
    bz = prob.bface[o:o + (N0[2] + 1) * N0[1] * N0[0]].reshape(N0[2] + 1, N0[1], N0[0])
    bf = inputs.pack_faces(bx[:nz, :ny, :nx + 1], by[:nz, :ny + 1, :nx], bz[:nz + 1, :ny, :nx])
    return inputs.Problem(name=prob.name + "_crop", n=n, x0=prob.x0, dx=prob.dx, prims=prims, bface=bf)


def test_parity_noise_box(orc):
    """Seeded white noise in every primitive: most MP5 reconstructions fail
    the monotonicity test, so the limiter's packed lists run long (in FP64
    up to 16 items per thread, 2048 per block of 128) -- L(U) on a ragged
    grid to 1e-12 and two steps to 1e-11 against the oracle."""
    from paper_1810_04597_gb300.echo import Solver
    base = crop(inputs.smooth_box(40, seed=13), (37, 29, 23))
    rng = np.random.default_rng(2024)
    shape = (base.n[2], base.n[1], base.n[0])
    prims = np.stack([rng.uniform(0.5, 1.5, shape), rng.uniform(-0.3, 0.3, shape), rng.uniform(-0.3, 0.3, shape),
                      rng.uniform(-0.3, 0.3, shape), rng.uniform(0.5, 1.5, shape)])
    prob = inputs.Problem(name="noise_box", n=base.n, x0=base.x0, dx=base.dx, prims=prims, bface=base.bface)
    s = Solver(prob)
    s.set_prims()
    L_g = s.rhs()
    cfg = orc.make_cfg(prob)
    st, Z = orc.p2c(cfg, prob.prims, prob.bface)
    L_o, _, _ = orc.rhs(cfg, st, Z)
    errs = per_field(orc, L_g, L_o, prob.n)
    assert max(errs.values()) <= 1e-12, errs
    st_g, _ = gpu_run(prob, 2)
    st_o, _, _, _ = oracle_run(orc, prob, 2)
    errs = per_field(orc, st_g, st_o, prob.n)
    assert max(errs.values()) <= 1e-11, errs


def test_ten_step_parity_32(orc):
    """The FP64 target: 10 steps of the 32^3 box, max-relative error per
    field <= 1e-11, CFL dt from each side's own state."""
    prob = inputs.smooth_box(32)
    st_g, s = gpu_run(prob, 10)
    st_o, Z_o, dts, stats = oracle_run(orc, prob, 10)
    errs = per_field(orc, st_g, st_o, prob.n)
    assert max(errs.values()) <= 1e-11, errs
    tg = s.reduce()
    cfg = orc.make_cfg(prob)
    to = orc.reduce(cfg, st_o)
    assert abs(tg["mass"] - to[0]) <= 1e-13 * abs(to[0])
    assert abs(tg["energy"] - to[1]) <= 1e-13 * abs(to[1])
    assert tg["c2p_fail"] == 0


def test_parity_ragged_steps(orc):
    prob = crop(inputs.smooth_box(40, seed=11), (33, 21, 17))
    st_g, _ = gpu_run(prob, 3)
    st_o, _, _, _ = oracle_run(orc, prob, 3)
    errs = per_field(orc, st_g, st_o, prob.n)
    assert max(errs.values()) <= 1e-11, errs


@pytest.mark.parametrize("kind", ["1d", "2d"])
def test_parity_low_dimensional(orc, kind):
    prob = inputs.alfven_wave(48) if kind == "1d" else inputs.alfven_wave_2d(24)
    st_g, _ = gpu_run(prob, 5)
    st_o, _, _, _ = oracle_run(orc, prob, 5)
    errs = per_field(orc, st_g, st_o, prob.n)
    assert max(errs.values()) <= 1e-11, errs


def test_parity_relativistic_shear(orc):
    """Face states with v^2 >= 1 (a flow at |v| = 0.99 turning over two
    cells) fall back to their own side's cell on both paths; the face
    velocities after the fallback also feed the edge EMFs (B != 0).  One
    step: the inversion of this state fails within the second without
    floors."""
    prob = inputs.relativistic_shear(32, B=(0.1, 0.05, 0.02))
    st_g, s = gpu_run(prob, 1)
    st_o, _, _, stats = oracle_run(orc, prob, 1)
    assert stats["fallback_faces"] > 0
    # the same face sides were replaced on both paths (counted on the faces
    # that bound owned cells)
    assert s.counters()["fallback_faces"] == stats["fallback_faces"]
    errs = per_field(orc, st_g, st_o, prob.n)
    assert max(errs.values()) <= 1e-11, errs


def test_fixed_dt_matches(orc):
    prob = inputs.smooth_box(16, seed=3)
    st_g, _ = gpu_run(prob, 4, dt=1e-3)
    st_o, _, _, _ = oracle_run(orc, prob, 4, dt=1e-3)
    errs = per_field(orc, st_g, st_o, prob.n)
    assert max(errs.values()) <= 1e-12, errs


def test_steps_from_any_start_match_the_oracle(orc):
    """Newton decides the inversion: five steps with the cold start in every
    c2p (mode 2) match the oracle (which starts from the previous-stage Z)
    like the default start does, with more iterations per inversion; the
    iteration histogram accounts for every inversion."""
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.smooth_box(20, seed=21)
    st_o, _, _, _ = oracle_run(orc, prob, 5)
    mean = {}
    for mode in (0, 2):
        s = Solver(prob)
        s.set_prims()
        s.set_c2p_guess(mode)
        for _ in range(5):
            s.step()
        c = s.counters()
        errs = per_field(orc, s.get_state(), st_o, prob.n)
        assert max(errs.values()) <= 1e-11, (mode, errs)
        h = np.array(c["c2p_iter_hist"])
        assert h.sum() == c["c2p_calls"] and int(np.dot(np.arange(h.size), h)) == c["c2p_iters"]
        mean[mode] = c["c2p_iters"] / c["c2p_calls"]
    print("mean Newton iterations per inversion, previous Z / cold:", mean)
    assert mean[2] > mean[0] + 0.5, mean


def test_uniform_state_is_exact():
    prob = inputs.uniform_box((16, 8, 4))
    st0, _ = gpu_run(prob, 0)
    st3, _ = gpu_run(prob, 3)
    cells = st3[:5 * prob.ncells].reshape(5, -1)
    assert np.all(np.ptp(cells, axis=1) == 0.0)
    assert np.max(np.abs(st3 - st0)) <= 1e-15 * np.max(np.abs(st0))


def test_zero_field_and_rest(orc):
    """Degenerate states: B = 0 everywhere (EMFs vanish) and v = 0; the
    pressure follows the density so that momentum builds up."""
    prob = inputs.smooth_box(16, seed=9)
    prob.bface = np.zeros_like(prob.bface)
    prob.prims[1:4] = 0.0
    prob.prims[4] = prob.prims[0] ** (4.0 / 3.0)
    st_g, _ = gpu_run(prob, 2)
    st_o, _, _, _ = oracle_run(orc, prob, 2)
    for name, a, b in zip(FIELDS, fields(orc, st_g, prob.n), fields(orc, st_o, prob.n)):
        if name.startswith("B"):
            assert np.all(a == 0.0)
        else:
            assert max_rel(a, b) <= 1e-12, name


def test_bitwise_determinism():
    prob = inputs.smooth_box(24, seed=4)
    a, sa = gpu_run(prob, 3)
    b, sb = gpu_run(prob, 3)
    assert np.array_equal(a, b)
    assert sa.reduce() == sb.reduce()


def test_set_state_roundtrip():
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.smooth_box(12, seed=2)
    s = Solver(prob)
    s.set_prims()
    st = s.get_state()
    z = s.get_z()
    s2 = Solver(prob)
    s2.set_state(st, z)
    assert np.array_equal(s2.get_state(), st)
    assert np.array_equal(s2.get_z(), z)


def test_device_pointers_match_host():
    import torch
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.smooth_box(12, seed=6)
    s = Solver(prob)
    s.set_prims(torch.from_numpy(np.ascontiguousarray(prob.prims)).cuda(),
                torch.from_numpy(np.ascontiguousarray(prob.bface)).cuda())
    s.step()
    out = torch.empty(s.nstate, dtype=torch.float64, device="cuda")
    s.get_state(out)
    h, _ = gpu_run(prob, 1)
    assert np.array_equal(out.cpu().numpy(), h)


def test_small_workspace_rejected():
    import torch
    from paper_1810_04597_gb300 import _lib
    prob = inputs.smooth_box(8)
    g = _lib.echo_grid()
    for d in range(3):
        g.n[d] = 8
        g.dx[d] = 1 / 8
    ctx = _lib.echo_init(g, _lib.echo_metric(0, 0), _lib.echo_eos(4 / 3, 0, 0, 0, 0, 0), 64, 0.4)
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(_lib.EchoError) as e:
        _lib.echo_bind(ctx, ws.data_ptr(), 1024, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == _lib.ECHO_ENOMEM
    _lib.echo_destroy(ctx)


def test_mapped_host_buffers_match_staged_copies():
    """on_device = 2: page-locked host buffers read and written by the
    kernels directly give the same state, primitives, Z and L(U) as the
    staged copies of plain host arrays; pageable memory is refused."""
    import ctypes
    import torch
    from paper_1810_04597_gb300 import _lib
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.smooth_box(20, seed=17)
    a = Solver(prob)
    a.set_prims()
    a.step()
    st = a.get_state()
    z = a.get_z()
    b = Solver(prob)
    st_p = torch.from_numpy(st.copy()).pin_memory()
    z_p = torch.from_numpy(z.copy()).pin_memory()
    b.set_state(st_p, z_p)
    out = torch.zeros(b.nstate, dtype=torch.float64).pin_memory()
    b.get_state(out)
    assert np.array_equal(out.numpy(), st)
    zo = torch.zeros(prob.ncells, dtype=torch.float64).pin_memory()
    b.get_z(zo)
    assert np.array_equal(zo.numpy(), z)
    L1 = a.rhs()
    Lp = torch.zeros(a.nstate, dtype=torch.float64).pin_memory()
    b.rhs(Lp)
    assert np.array_equal(Lp.numpy(), L1)
    plain = np.zeros(b.nstate)
    rc = _lib.load().echo_get_state(b.ctx, ctypes.c_void_p(plain.ctypes.data), 2)
    assert rc == _lib.ECHO_EINVAL
    rc = _lib.load().echo_get_state(b.ctx, ctypes.c_void_p(plain.ctypes.data), 3)
    assert rc == _lib.ECHO_EINVAL


def _inadmissible(orc, prob, cell):
    """The p2c state of prob with tau = -10 D in one cell: tau + D < 0 admits
    no Z > 0, so that inversion fails on both paths."""
    cfg = orc.make_cfg(prob)
    st, Z = orc.p2c(cfg, prob.prims, prob.bface)
    N = prob.ncells
    bad = st.copy()
    bad[4 * N + cell] = -10.0 * bad[cell]
    return cfg, bad, Z


def test_inadmissible_state_returns_ec2p(orc):
    """Floors off: a host-built state with one inadmissible cell makes
    echo_c2p return ECHO_EC2P with that one failure counted (the oracle
    fails on the same cell), and a step followed by echo_reduce reports it
    too."""
    from paper_1810_04597_gb300 import _lib
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.smooth_box(12, seed=5)
    cfg, bad, Z = _inadmissible(orc, prob, cell=123)
    _, _, ostats, orc_rc = orc.c2p(cfg, bad, Z, check=False)
    assert orc_rc != 0 and ostats["fails"] == 1
    s = Solver(prob)
    s.set_state(bad, Z)
    t = _lib.echo_totals()
    with pytest.raises(_lib.EchoError) as e:
        _lib.echo_c2p(s.ctx, 0, t)
    assert e.value.code == _lib.ECHO_EC2P
    assert t.c2p_fail == 1 and t.c2p_calls == prob.ncells
    s2 = Solver(prob)
    s2.set_state(bad, Z)
    s2.step(1e-4)
    with pytest.raises(_lib.EchoError) as e:
        s2.reduce()
    assert e.value.code == _lib.ECHO_EC2P
    # the error is reported once: a clean state afterwards reduces normally
    st, _ = orc.p2c(cfg, prob.prims, prob.bface)
    s2.set_state(st, Z)
    assert s2.reduce()["c2p_fail"] >= 1
