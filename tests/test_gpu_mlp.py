"""The c2p-guess network on the GPU: forward pass and batch gradient against
the FP64 oracle, the Adam update, training on method-generated pairs, and
what the trained guess gains (or loses) against the guesses without it."""
import numpy as np
import pytest

from paper_1810_04597_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return T


def random_state(T, rng):
    from paper_1810_04597_gb300 import _lib
    st = np.zeros(_lib.ECHO_MLP_STATE, dtype=np.float32)
    st[:4995] = rng.normal(0, 0.3, 4995)
    st[4995:4995 + 9] = rng.normal(0, 1, 9)
    st[4995 + 9:4995 + 18] = rng.uniform(0.5, 2, 9)
    st[4995 + 18:4995 + 21] = rng.normal(0, 0.5, 3)
    st[4995 + 21:4995 + 24] = rng.uniform(0.5, 2, 3)
    return st


def random_rows(rng, n):
    x = rng.normal(0, 1, size=(n, 9)).astype(np.float32)
    W = rng.uniform(1.0, 1.5, n)
    pD = rng.uniform(0.1, 2.0, n)
    z = W * (1 + 4.0 * pD * W)
    y = np.stack([np.log(W), np.log(pD), np.log(z)], axis=1).astype(np.float32)
    return x, y


def test_forward_matches_oracle(orc, torch):
    from paper_1810_04597_gb300 import _lib
    rng = np.random.default_rng(0)
    st = random_state(torch, rng)
    x, _ = random_rows(rng, 1000)
    out = torch.empty((1000, 3), dtype=torch.float32, device="cuda")
    _lib.echo_mlp_forward(torch.from_numpy(st).cuda(), torch.from_numpy(x).cuda(), 1000, out)
    ref = orc.mlp_forward(st[:4995 + 24].astype(np.float64), x.astype(np.float64))
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 2e-5 * max(1.0, np.max(np.abs(ref)))


def test_gradient_matches_oracle(orc, torch):
    from paper_1810_04597_gb300 import _lib
    rng = np.random.default_rng(1)
    st = random_state(torch, rng)
    x, y = random_rows(rng, 2048)
    batch = 2048
    g = torch.empty(4995, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    work = torch.empty(_lib.echo_mlp_work_bytes(batch), dtype=torch.uint8, device="cuda")
    _lib.echo_mlp_grad(torch.from_numpy(st).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                       2048, 0, batch, 4.0 / 3.0, g, loss, work)
    lo, go = orc.mlp_loss_grad(st[:4995 + 24].astype(np.float64), x.astype(np.float64), y.astype(np.float64),
                               w2=0.1)
    gg = g.cpu().numpy().astype(np.float64)
    # element by element, against the largest gradient of the parameter's own
    # block (W1, b1, W2, b2, W3, b3), so that small blocks such as the biases
    # and the output layer are checked at their own scale
    bounds = [0, 576, 640, 4736, 4800, 4992, 4995]
    for a, b in zip(bounds[:-1], bounds[1:]):
        scale = np.max(np.abs(go[a:b]))
        assert scale > 0.0
        worst = np.max(np.abs(gg[a:b] - go[a:b])) / scale
        assert worst <= 1e-4, (a, b, worst)
    assert abs(float(loss.item()) - lo) <= 1e-4 * abs(lo)


def test_adam_step_matches_oracle(orc, torch):
    from paper_1810_04597_gb300 import _lib
    rng = np.random.default_rng(2)
    st = random_state(torch, rng)
    x, y = random_rows(rng, 512)
    dst = torch.from_numpy(st.copy()).cuda()
    work = torch.empty(_lib.echo_mlp_work_bytes(512), dtype=torch.uint8, device="cuda")
    _lib.echo_mlp_train(dst, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 512, 512, 1, 0, 1e-3,
                        4.0 / 3.0, work)
    _, go = orc.mlp_loss_grad(st[:4995 + 24].astype(np.float64), x.astype(np.float64), y.astype(np.float64),
                              w2=0.1)
    P = st[:4995].astype(np.float64)
    m = np.zeros(4995)
    v = np.zeros(4995)
    orc.mlp_adam(P, m, v, go, 1, lr=1e-3)
    got = dst.cpu().numpy()[:4995].astype(np.float64)
    # the first Adam step is lr * sign(g) per parameter: compare the move
    moved = got - st[:4995]
    ref = P - st[:4995]
    big = np.abs(go) > 1e-3 * np.max(np.abs(go))
    assert np.allclose(moved[big], ref[big], rtol=1e-3, atol=1e-7)


@pytest.fixture(scope="module")
def trained(torch):
    from paper_1810_04597_gb300 import mlp
    runs = [(inputs.sweep_box(64), [0, 2, 4, 6, 8]), (inputs.smooth_box(64), [0, 3, 6])]
    (Xtr, Ytr), (Xva, Yva), (Xte, Yte) = mlp.collect(runs)
    state, losses = mlp.train(Xtr, Ytr, epochs=3, batch=4096, lr=2e-3)
    mlp.calibrate(state, Xva, Yva)
    return state, losses, (Xte, Yte)


def test_training_reduces_loss_and_error(trained, torch):
    from paper_1810_04597_gb300 import mlp
    state, losses, (Xte, Yte) = trained
    L = losses.cpu().numpy()
    assert np.all(np.isfinite(L))
    assert L[-50:].mean() < 0.05 * L[:20].mean(), (L[:20].mean(), L[-50:].mean())
    err = mlp.guess_error(state, Xte, Yte).cpu().numpy()
    assert np.median(err) < 1e-2, np.median(err)
    # the library's error against its definition written out here: the start
    # Z0 / D = W (1 + G/(G-1) (p/D) W) from the de-standardised outputs
    from paper_1810_04597_gb300 import _lib
    n = Xte.shape[0]
    out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    _lib.echo_mlp_forward(state, Xte, n, out, torch.cuda.current_stream().cuda_stream)
    blk = state[:_lib.ECHO_MLP_BLOCK].double().cpu().numpy()
    ym, ys = blk[4995 + 18:4995 + 21], blk[4995 + 21:4995 + 24]
    o = out.double().cpu().numpy() * ys + ym
    W = np.exp(o[:, 0])
    z0 = W * (1.0 + 4.0 * np.exp(o[:, 1]) * W)
    z = np.exp(Yte[:, 2].double().cpu().numpy())
    want = np.abs(z0 - z) / z
    assert np.allclose(err, want, rtol=1e-5, atol=1e-7)
    # the tensor-core forward c2p uses (BF16 operands, hardware tanh)
    err_tc = mlp.guess_error(state, Xte, Yte, tensor_cores=True).cpu().numpy()
    print("held-out guess error, median: FP32", np.median(err), "tensor cores", np.median(err_tc))
    assert np.median(err_tc) < 1.5e-2, np.median(err_tc)


def _cold(s):
    """Restart s from its own state without the Newton memory: every tile is
    flagged and every cell's previous Z is cold, so the network is consulted
    everywhere."""
    st = s.get_state()
    s.set_state(st)
    return st


def test_network_guess_gives_the_same_inversion(trained, torch):
    """The Newton solve stays the judge: from a cold restart the network
    start is taken by (nearly) every cell, and the converged primitives equal
    those from the cold start without the network to rounding."""
    from paper_1810_04597_gb300.echo import Solver
    state, _, _ = trained
    prob = inputs.sweep_box(48, seed=77)
    a = Solver(prob)
    a.set_prims()
    b = Solver(prob)
    b.set_prims()
    b.mlp_load(state)
    a.step()
    b.step()
    _cold(a)
    _cold(b)
    sa = a.c2p(2)
    c0 = b.counters()
    sb = b.c2p(1)
    Pa = a.get_prims()
    Pb = b.get_prims()
    for q in range(8):
        assert np.max(np.abs(Pa[q] - Pb[q])) <= 1e-12 * max(np.max(np.abs(Pa[q])), 1e-300), q
    assert sb["mlp_used"] - c0["mlp_used"] >= 0.9 * prob.ncells
    assert sb["mlp_fallback"] <= 0.01 * prob.ncells


def test_gain_over_guesses_without_network(trained, torch):
    """Mean Newton iterations per c2p call during three SSP-RK3 steps with
    the previous-stage guess and with the network guess (chosen per cell),
    and for one inversion from the cold guess, on a held-out input.  In a
    time-stepping run the previous Z is usually the closer start, so the
    per-cell choice must do at least as well as it (within rounding of the
    mean) and beat the cold guess, and reproduce the same state; from a cold
    restart the network must beat the cold guess."""
    from paper_1810_04597_gb300.echo import Solver
    state, _, _ = trained
    prob = inputs.sweep_box(64, seed=99)
    res, fin = {}, {}
    for mode, name in ((0, "previous"), (1, "network")):
        s = Solver(prob)
        s.set_prims()
        s.mlp_load(state)
        s.set_c2p_guess(mode)
        c0 = s.counters()
        for _ in range(3):
            s.step()
        c1 = s.counters()
        res[name] = (c1["c2p_iters"] - c0["c2p_iters"]) / (c1["c2p_calls"] - c0["c2p_calls"])
        res[name + "_fallback"] = c1["mlp_fallback"] - c0["mlp_fallback"]
        fin[name] = s.get_state()
    s = Solver(prob)
    s.set_prims()
    c0 = s.counters()
    s.c2p(2)
    c1 = s.counters()
    res["cold"] = (c1["c2p_iters"] - c0["c2p_iters"]) / (c1["c2p_calls"] - c0["c2p_calls"])
    # cold restart: the network start against the cold guess
    for mode, name in ((2, "restart_cold"), (1, "restart_network")):
        s = Solver(prob)
        s.set_prims()
        s.mlp_load(state)
        s.step()
        _cold(s)
        c0 = s.counters()
        s.c2p(mode)
        c1 = s.counters()
        res[name] = (c1["c2p_iters"] - c0["c2p_iters"]) / (c1["c2p_calls"] - c0["c2p_calls"])
    print("mean Newton iterations per call:", res)
    assert res["network"] < res["cold"]
    assert res["network"] <= res["previous"] + 0.01, res
    assert res["restart_network"] < res["restart_cold"] - 0.5, res
    scale = np.max(np.abs(fin["previous"]))
    assert np.max(np.abs(fin["network"] - fin["previous"])) <= 1e-11 * scale


def test_refined_gate_lists_only_large_moves(trained, torch):
    """With the FP32 refinement (mode 5) a cell is listed only where its Z
    moved by about 1/8 or more, since the refinement brings any closer start
    to the same single FP64 iteration: in a smooth FP32 run far fewer cells
    start from the network than without the refinement (mode 1, the plain
    gate), the FP64 iterations stay at those of the previous-Z start, and the
    state equals the previous-Z run's to FP32 rounding (relative L1).  Changing the
    refinement flag empties the list: the first inversion after the change
    starts no cell from the network."""
    from paper_1810_04597_gb300.echo import Solver
    state, _, _ = trained
    prob = inputs.sweep_box(48, seed=93)
    res, fin = {}, {}
    for mode in (4, 5, 1):
        s = Solver(prob, precision=32)
        s.set_prims()
        s.mlp_load(state)
        s.set_c2p_guess(mode)
        for _ in range(2):
            s.step()
        c0 = s.counters()
        for _ in range(3):
            s.step()
        c1 = s.counters()
        calls = c1["c2p_calls"] - c0["c2p_calls"]
        res[mode] = ((c1["c2p_iters"] - c0["c2p_iters"]) / calls, (c1["mlp_used"] - c0["mlp_used"]) / calls,
                     c1["mlp_fallback"] - c0["mlp_fallback"])
        fin[mode] = s.get_state()
        if mode == 5:
            # the refinement flag changes: the list made under the refined gate is dropped
            c2 = s.counters()
            s.c2p(1)
            c3 = s.counters()
            res["switch"] = c3["mlp_used"] - c2["mlp_used"]
    print("FP32 (mean FP64 its, network starts per cell, fallbacks): previous Z", res[4], "refined gate", res[5],
          "plain gate", res[1], "starts after the switch", res["switch"])
    assert res[1][1] > 0.0, res
    assert res[5][1] <= 0.2 * res[1][1], res
    assert res[5][0] <= res[4][0] + 0.005, res
    assert res[5][2] == 0 and res["switch"] == 0, res
    # Newton decides: the same state to FP32 rounding (relative L1)
    assert np.sum(np.abs(fin[5] - fin[4])) <= 1e-6 * np.sum(np.abs(fin[4]))


def _bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _forward_bf16_hidden(st, x):
    """FP64 forward pass with the tensor-core operands rounded as the GPU
    rounds them: the standardised features (FP32, times 1/std in FP32), W1,
    h1 (from FP32) and W2 to BF16; raw outputs."""
    P = st.astype(np.float64)
    mu, sd = P[4995:5004], P[5004:5013]
    W1, b1 = P[0:576].reshape(64, 9), P[576:640]
    W2, b2 = P[640:4736].reshape(64, 64), P[4736:4800]
    W3, b3 = P[4800:4992].reshape(3, 64), P[4992:4995]
    isd = (np.float32(1.0) / sd.astype(np.float32)).astype(np.float32)
    xs = _bf16((x.astype(np.float32) - mu.astype(np.float32)) * isd)
    h1 = _bf16(np.tanh(xs @ _bf16(W1.astype(np.float32)).T + b1).astype(np.float32))
    h2 = np.tanh(h1 @ _bf16(W2.astype(np.float32)).T + b2)
    return h2 @ W3.T + b3


def test_tensor_core_forward(orc, torch):
    """Both hidden layers on the tensor cores (tcgen05, BF16 operands, FP32
    accumulation) match the FP64 forward pass with the same BF16 roundings
    to the accuracy of the hardware tanh; ragged last tile included."""
    from paper_1810_04597_gb300 import _lib
    rng = np.random.default_rng(3)
    st = random_state(torch, rng)
    n = 4099
    x, _ = random_rows(rng, n)
    dst, dx = torch.from_numpy(st).cuda(), torch.from_numpy(x).cuda()
    out = torch.full((n, 3), -7.0, dtype=torch.float32, device="cuda")
    _lib.echo_mlp_forward_tc(dst, dx, n, out)
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    emu = _forward_bf16_hidden(st[:4995 + 24], x)
    d = np.abs(got - emu)
    print("tensor-core forward vs BF16 model: median", np.median(d), "max", np.max(d))
    # the kernel's tanh is the hardware approximation (relative error about
    # 2^-11), which also flips some BF16 roundings of h1 (measured: median
    # 4e-6, max 5e-3 on outputs of order one); a wrong operand layout or
    # descriptor gives errors of order one
    assert np.median(d) <= 2e-5 and np.max(d) <= 1.5e-2, (np.median(d), np.max(d))
    ref = orc.mlp_forward(st[:4995 + 24].astype(np.float64), x.astype(np.float64))
    print("tensor-core forward: max |tc - fp64| =", np.max(np.abs(got - ref)), " max |tc - bf16 model| =", d.max())


@pytest.mark.parametrize("precision,modes", [(64, (9, 1, 17)), (32, (13, 5, 21))])
def test_tensor_core_guess_gives_the_same_inversion(trained, torch, precision, modes):
    """c2p from a cold restart with the network guess evaluated on the CUDA
    cores, on the tensor cores in a pass of its own, and on the tensor cores
    inside the c2p kernel (every tile flagged, nearly every cell taking the
    network start):
    Newton decides, so the primitives agree (FP64: to 1e-12; FP32 storage: to
    its rounding), with no fallback; the two tensor-core forms give the same
    starts and the same iterations."""
    from paper_1810_04597_gb300.echo import Solver
    state, _, _ = trained
    prob = inputs.sweep_box(41, seed=78)          # 68,921 cells: a ragged last tile
    out = []
    for m in modes:
        s = Solver(prob, precision=precision)
        s.set_prims()
        s.mlp_load(state)
        s.step()
        _cold(s)
        c0 = s.counters()
        s.c2p(m)
        c1 = s.counters()
        assert c1["mlp_used"] - c0["mlp_used"] >= 0.9 * prob.ncells, m
        out.append((s.get_prims(), s.get_z(), c1["mlp_fallback"] - c0["mlp_fallback"],
                    (c1["c2p_iters"] - c0["c2p_iters"]) / (c1["c2p_calls"] - c0["c2p_calls"])))
    (Pa, Za, fa, ia) = out[0]
    tol = 1e-12 if precision == 64 else 2.5e-7
    for (Pb, Zb, fb, ib) in out[1:]:
        assert fb == 0 and fa == 0
        assert np.max(np.abs(Za - Zb) / Za) <= (1e-12 if precision == 64 else 1e-10)
        for q in range(5):
            assert np.max(np.abs(Pa[q] - Pb[q])) <= tol * max(np.max(np.abs(Pa[q])), 1e-300), q
        assert abs(ia - ib) <= 0.5
    print(f"precision {precision}: Newton iterations per call, CUDA-core guess {ia:.3f}, tensor-core guess "
          f"{out[1][3]:.3f} (own pass), {out[2][3]:.3f} (inside c2p)")
    # same starts; the two kernels may contract multiply-adds differently
    assert abs(out[1][3] - out[2][3]) <= 1e-3
    for q in range(5):
        assert np.max(np.abs(out[1][0][q] - out[2][0][q])) <= 1e-13 * max(np.max(np.abs(out[1][0][q])), 1e-300), q


def test_torus_training_reduces_fallbacks(torch):
    """A network trained on the periodic boxes alone meets states it never saw
    in a torus atmosphere (tiny density, high magnetisation); adding torus
    snapshots to the training data must cut the fallbacks to the previous-
    stage guess and the Newton iterations of a cold restart of a held-out
    torus (spin 0.5, another seed, after 6 steps).  Fallbacks are counted net
    of the cells whose inversion fails from every guess (those end at the
    floors either way).  In the running torus, the per-cell choice with the
    torus-trained network needs no more Newton iterations than the plain
    previous-stage start, with no more fallbacks than failures."""
    from paper_1810_04597_gb300 import mlp
    from paper_1810_04597_gb300.echo import Solver
    nets = {"box": mlp.default_network(n=64)[0], "box+torus": mlp.default_network(n=64, torus=True)[0]}
    prob = inputs.fm_torus((96, 48, 48), spin=0.5, beta=30.0, seed=inputs.SEED_BASE + 299)
    res = {}
    for name, state in nets.items():
        s = Solver(prob)
        s.set_prims()
        s.mlp_load(state)
        for _ in range(6):
            s.step()
        _cold(s)
        c0 = s.counters()
        s.c2p(1)
        c1 = s.counters()
        calls = c1["c2p_calls"] - c0["c2p_calls"]
        soft = (c1["mlp_fallback"] - c0["mlp_fallback"]) - (c1["c2p_fail"] - c0["c2p_fail"])
        res[name] = (soft / calls, (c1["c2p_iters"] - c0["c2p_iters"]) / calls)
    run = {}
    for mode in (0, 1):
        s = Solver(prob)
        s.set_prims()
        s.mlp_load(nets["box+torus"])
        s.set_c2p_guess(mode)
        c0 = s.counters()
        for _ in range(6):
            s.step()
        c1 = s.counters()
        calls = c1["c2p_calls"] - c0["c2p_calls"]
        run[mode] = ((c1["c2p_iters"] - c0["c2p_iters"]) / calls, (c1["mlp_used"] - c0["mlp_used"]) / calls,
                     c1["mlp_fallback"] - c0["mlp_fallback"], c1["c2p_fail"] - c0["c2p_fail"])
    print("held-out torus, cold restart: (fallbacks per call, Newton iterations per call):", res)
    print("running torus (iterations per call, network starts per call, fallbacks, failures): previous Z",
          run[0], "per-cell choice", run[1])
    assert res["box+torus"][0] <= res["box"][0], res
    assert res["box+torus"][1] < 0.9 * res["box"][1], res
    assert run[1][0] <= run[0][0] + 0.005, run


@pytest.mark.parametrize("kind", ["box", "torus"])
def test_dataset_rows_match_their_definitions(orc, torch, kind):
    """echo_mlp_dataset's nine features and three targets, element by
    element, against their definitions written out here in numpy (FP64) on
    the same conserved state: metric from the oracle's closed form at the
    cell centres, cell-centre B the mean of the two faces over sqrt(gamma),
    targets from the oracle's converged inversion; cell c lands in row
    (c * 2654435761) mod N."""
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.sweep_box(12, seed=55) if kind == "box" else inputs.fm_torus((24, 12, 6), seed=57)
    s = Solver(prob)
    s.set_prims()
    N = prob.ncells
    X = torch.empty((N, 9), dtype=torch.float32, device="cuda")
    Y = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    s.mlp_dataset(X, Y)
    st = s.get_state()       # after the dataset's own c2p (floors may reset cells)
    Xg, Yg = X.cpu().numpy().astype(np.float64), Y.cpu().numpy().astype(np.float64)
    cfg = orc.make_cfg(prob)
    P_o, Z_o, _, _ = orc.c2p(cfg, st, s.get_z(), check=False)
    nx, ny, nz = prob.n
    cells, bx, by, bz = orc.split_state(st, prob.n)
    Bt = np.stack([0.5 * (bx[:, :, :-1] + bx[:, :, 1:]), 0.5 * (by[:, :-1, :] + by[:, 1:, :]),
                   0.5 * (bz[:-1] + bz[1:])]).reshape(3, -1)
    U = cells.reshape(5, -1)
    ref = np.zeros((N, 9))
    tgt = np.zeros((N, 3))
    for c in range(N):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        x = [prob.x0[0] + (i + 0.5) * prob.dx[0], prob.x0[1] + (j + 0.5) * prob.dx[1],
             prob.x0[2] + (k + 0.5) * prob.dx[2]]
        m = orc.metric_point(cfg, x)
        sg = m["sqrtg"]
        D, S, tau, B = U[0, c] / sg, U[1:4, c] / sg, U[4, c] / sg, Bt[:, c] / sg
        S2 = S @ m["gi"] @ S
        B2 = B @ m["g"] @ B
        SB = S @ B
        ref[c] = [np.log(max(tau / D, 1e-30)), np.log1p(S2 / D ** 2), np.log1p(B2 / D),
                  SB ** 2 / (S2 * B2 + 1e-30), m["alpha"], np.log(sg), m["beta"] @ m["g"] @ m["beta"],
                  np.trace(m["gi"]) / 3.0, np.clip(np.log(D), -30.0, 30.0) / 10.0]
        v = P_o[1:4, c]
        W = 1.0 / np.sqrt(1.0 - v @ m["g"] @ v)
        tgt[c] = [np.log(W), np.log(P_o[4, c] / D), np.log(Z_o[c] / D)]
    rows = (np.arange(N, dtype=np.uint64) * np.uint64(2654435761)) % np.uint64(N)
    assert len(set(rows.tolist())) == N
    got_f, got_t = Xg[rows.astype(np.int64)], Yg[rows.astype(np.int64)]
    for q in range(9):
        assert np.allclose(got_f[:, q], ref[:, q], rtol=2e-5, atol=2e-5), (q, np.max(np.abs(got_f[:, q] - ref[:, q])))
    for q in range(3):
        assert np.allclose(got_t[:, q], tgt[:, q], rtol=1e-6, atol=1e-6), (q, np.max(np.abs(got_t[:, q] - tgt[:, q])))
