"""Batch of independent runs under each schedule (persistent cooperative
kernel per RK stage, one launch per phase, run-major with concurrent
branches): the same results as the runs advanced one at a time -- bitwise
for run-major (the same kernels), to rounding for the other two (the same
device bodies compiled into other kernels) -- with and without CUDA-graph
replay."""
import numpy as np
import pytest

from paper_1810_04597_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _tori(precision=64):
    from paper_1810_04597_gb300.echo import Solver
    probs = [inputs.fm_torus((32, 16, 8), spin=0.5, seed=1), inputs.fm_torus((48, 24, 8), spin=0.9, seed=2),
             inputs.fm_torus((40, 20, 12), spin=0.0, beta=10.0, seed=3)]
    out = []
    for p in probs:
        s = Solver(p, precision=precision)
        s.set_prims()
        out.append(s)
    return out


@pytest.mark.parametrize("tile,dyn,graph,mode,branches", [
    (256, True, False, 0, 1), (128, False, False, 0, 1), (512, True, True, 0, 1), (256, True, False, 1, 1),
    (1024, True, True, 1, 1), (256, True, False, 2, 1), (256, True, True, 2, 1), (256, True, False, 2, 2),
    (256, True, True, 2, 3)])
def test_batch_equals_runs_one_at_a_time(tile, dyn, graph, mode, branches):
    from paper_1810_04597_gb300.batch import Batch
    single = _tori()
    for s in single:
        for _ in range(3):
            s.step()
    ref = [s.get_state() for s in single]
    runs = _tori()
    b = Batch(runs)
    b.configure(tile=tile, dynamic=dyn, mode=mode, branches=branches)
    b.graph(graph)
    for _ in range(3):
        b.step()
    for r, s in zip(ref, runs):
        got = s.get_state()
        if mode == 2:
            # run-major runs the single-run kernels themselves: bitwise
            assert np.array_equal(got, r), np.max(np.abs(got - r))
        else:
            # the persistent and per-phase kernels compile the same device code
            # in other kernels; ptxas may fuse a multiply and an add into one
            # FMA differently there, so they agree to rounding, not bitwise
            assert np.max(np.abs(got - r)) <= 1e-12 * np.max(np.abs(r)), np.max(np.abs(got - r))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_matches_the_oracle(orc, mode):
    """Each of the three uneven tori advanced by the batch (FP64) under each
    schedule matches the oracle's own run of that torus after 10 steps to
    1e-11 per field (CFL dt per run)."""
    from paper_1810_04597_gb300.batch import Batch
    from gpu_util import oracle_run, per_field
    runs = _tori()
    probs = [s.problem for s in runs]
    b = Batch(runs)
    b.configure(mode=mode, branches=2 if mode == 2 else 1)
    for _ in range(10):
        b.step()
    for s, p in zip(runs, probs):
        st_o, _, _, _ = oracle_run(orc, p, 10)
        errs = per_field(orc, s.get_state(), st_o, p.n)
        assert max(errs.values()) <= 1e-11, (p.n, errs)


def test_batch_flat_fixed_dt_and_counters():
    from paper_1810_04597_gb300.batch import Batch
    from paper_1810_04597_gb300.echo import Solver
    probs = [inputs.smooth_box(16, seed=s) for s in (1, 2)] + [inputs.sweep_box(24, seed=3)]
    a = [Solver(p) for p in probs]
    c = [Solver(p) for p in probs]
    for s in a + c:
        s.set_prims()
    for s in a:
        s.step(1e-3)
        s.step(1e-3)
    b = Batch(c)
    b.step(1e-3)
    b.step(1e-3)
    for x, y in zip(a, c):
        sx, sy = x.get_state(), y.get_state()
        assert np.max(np.abs(sx - sy)) <= 1e-12 * np.max(np.abs(sx))
        assert x.counters()["c2p_calls"] == y.counters()["c2p_calls"]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_with_network_guess(mode):
    """FP32 tori from cold restarts with the network Newton start (guess 5)
    under each schedule.
    Run-major runs the single-run kernels: bitwise.  The persistent and
    per-phase schedules take the starts from their own tensor-core pass over
    all runs (the persistent one before the stage's ghost fill, so a cell at
    a periodic seam may start from a field one stage old) and compile c2p
    into other kernels: the same converged inversions, states equal to the
    FP32 store's rounding."""
    import torch
    from paper_1810_04597_gb300.batch import Batch
    rng = np.random.default_rng(77)
    from test_gpu_mlp import random_state
    state = torch.from_numpy(random_state(torch, rng)).cuda()
    single = _tori(32)
    runs = _tori(32)
    for s in single + runs:
        s.set_state(s.get_state())    # cold restarts: every tile consults the network first
        s.mlp_load(state)
        s.set_c2p_guess(5)
    for s in single:
        for _ in range(2):
            s.step()
    b = Batch(runs)
    b.configure(mode=mode, branches=2 if mode == 2 else 1)
    for _ in range(2):
        b.step()
    for s, r in zip(runs, single):
        got, ref = s.get_state(), r.get_state()
        assert np.all(np.isfinite(got))
        if mode == 2:
            assert np.array_equal(got, ref), np.max(np.abs(got - ref))
        else:
            # a floor decision can flip with the last FP32 bit of a cell: L1
            # to the store's rounding, max loosely
            l1 = np.sum(np.abs(got - ref)) / np.sum(np.abs(ref))
            assert l1 <= 1e-6, l1
            assert np.max(np.abs(got - ref)) <= 1e-3 * np.max(np.abs(ref)), np.max(np.abs(got - ref))
