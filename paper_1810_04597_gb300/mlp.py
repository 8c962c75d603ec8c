"""Training driver of the c2p-guess network (orchestration only).

Data: converged inversions the method itself produces -- every owned cell of
FP64 runs of the periodic boxes (``sweep_box``, ``smooth_box``), a few
snapshots along each run, written by ``echo_mlp_dataset`` in a permuted cell
order and interleaved across snapshots.  Training: ``echo_mlp_normalize`` and
``echo_mlp_train`` (Adam) -- every forward, backward and update runs in the
library's kernels.  Torch only supplies device memory and the stream.
"""
from __future__ import annotations

from . import _lib, inputs
from .echo import Solver


def collect(problems_and_steps, device="cuda:0"):
    """Snapshots -> (X, Y) train / validation / test tensors on `device`.

    problems_and_steps: list of (problem, [steps at which to take a
    snapshot]).  In every run the last snapshot is held out for test, the one
    before it for validation, the others train (rows interleaved across the
    training snapshots, or shuffled when the snapshots differ in size)."""
    import torch
    train_s, val_s, test_s = [], [], []
    for prob, at in problems_and_steps:
        at = sorted(at)
        s = Solver(prob, precision=64, device=device)
        s.set_prims()
        snaps = []
        for step in range(at[-1] + 1):
            if step in at:
                N = prob.ncells
                X = torch.empty((N, 9), dtype=torch.float32, device=device)
                Y = torch.empty((N, 3), dtype=torch.float32, device=device)
                s.mlp_dataset(X, Y, 0, 1)
                snaps.append((X, Y))
            if step < at[-1]:
                s.step()
        s.close()
        train_s += snaps[:-2]
        val_s.append(snaps[-2])
        test_s.append(snaps[-1])
    sizes = {x.shape[0] for x, _ in train_s}
    if len(sizes) == 1:
        Xtr = torch.stack([x for x, _ in train_s], dim=1).reshape(-1, 9).contiguous()
        Ytr = torch.stack([y for _, y in train_s], dim=1).reshape(-1, 3).contiguous()
    else:
        # snapshots of different sizes: all rows, in a fixed pseudo-random order
        Xtr = torch.cat([x for x, _ in train_s], dim=0)
        Ytr = torch.cat([y for _, y in train_s], dim=0)
        g = torch.Generator(device="cpu").manual_seed(12345)
        perm = torch.randperm(Xtr.shape[0], generator=g).to(Xtr.device)
        Xtr, Ytr = Xtr[perm].contiguous(), Ytr[perm].contiguous()
    cat = lambda xs: torch.cat(xs, dim=0).contiguous()  # noqa: E731
    return (Xtr, Ytr), (cat([x for x, _ in val_s]), cat([y for _, y in val_s])), \
        (cat([x for x, _ in test_s]), cat([y for _, y in test_s]))


def calibrate(state, X, Y, gamma=4.0 / 3.0):
    """Set the network's gate (the mean log10 error of its Newton starts on
    rows (X, Y), ``echo_mlp_calibrate``): cells whose previous-stage Z moved
    less than that do not consult the network."""
    import torch
    n = X.shape[0]
    out = torch.empty((n, 3), dtype=torch.float32, device=X.device)
    err = torch.empty(n, dtype=torch.float32, device=X.device)
    _lib.echo_mlp_calibrate(state, X, Y, n, gamma, out, err, torch.cuda.current_stream(X.device).cuda_stream)
    return float(state[_lib.ECHO_MLP_GATE].item())


def train(X, Y, epochs=2, batch=8192, lr=1e-3, seed=1, gamma=4.0 / 3.0, device="cuda:0"):
    """Train a fresh network on (X, Y); returns (state tensor, per-step
    losses tensor).  The gate is left at 0 (only cold starts consult the
    network) until ``calibrate``."""
    import torch
    n = X.shape[0]
    state = torch.empty(_lib.ECHO_MLP_STATE, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream(device).cuda_stream
    _lib.echo_mlp_init(state, seed, stream)
    work = torch.empty(_lib.echo_mlp_work_bytes(batch), dtype=torch.uint8, device=device)
    _lib.echo_mlp_normalize(state, X, Y, n, work, stream)
    nsteps = max(1, int(epochs * n // batch))
    losses = torch.empty(nsteps, dtype=torch.float32, device=device)
    chunk = 512
    for s0 in range(0, nsteps, chunk):
        k = min(chunk, nsteps - s0)
        _lib.echo_mlp_train(state, X, Y, n, batch, k, s0, lr, gamma, work, losses[s0:s0 + k], stream)
    return state, losses


def guess_error(state, X, Y, gamma=4.0 / 3.0, tensor_cores=False):
    """Relative error |Z0 - Z| / Z of the network guess on rows (X, Y),
    computed by the library (``echo_mlp_guess_error``): the FP32 CUDA-core
    forward, or with tensor_cores the BF16 tensor-core forward that c2p
    uses."""
    import torch
    n = X.shape[0]
    out = torch.empty((n, 3), dtype=torch.float32, device=X.device)
    err = torch.empty(n, dtype=torch.float32, device=X.device)
    _lib.echo_mlp_guess_error(state, X, Y, n, gamma, tensor_cores, out, err,
                              torch.cuda.current_stream(X.device).cuda_stream)
    return err


def box_runs(n=128):
    """Snapshots of FP64 runs of the two periodic boxes at n^3: the
    throughput recipe (sweep_box) and the parity recipe (smooth_box)."""
    return [(inputs.sweep_box(n), [0, 3, 6, 9, 12, 15]),
            (inputs.smooth_box(n), [0, 4, 8, 12])]


def torus_runs(n=(96, 48, 48)):
    """Snapshots of FP64 Fishbone-Moncrief torus runs on Kerr-Schild (spins
    0 and 0.9, beta 10 and 100): the atmosphere at the floors and the
    magnetised torus, where the box data do not reach."""
    runs = []
    for k, (spin, beta) in enumerate(((0.0, 10.0), (0.9, 100.0), (0.9, 10.0), (0.0, 100.0))):
        prob = inputs.fm_torus(n, spin=spin, beta=beta, seed=inputs.SEED_BASE + 200 + k)
        runs.append((prob, [0, 4, 8, 12, 16, 20]))
    return runs


def default_network(device="cuda:0", n=128, epochs=2, seed=1, torus=False):
    """The network used by the benchmarks: trained on snapshots of the n^3
    box runs (box_runs), and with torus=True also of the torus runs
    (torus_runs); its gate calibrated on the validation snapshots."""
    runs = box_runs(n) + (torus_runs() if torus else [])
    (Xtr, Ytr), (Xva, Yva), (Xte, Yte) = collect(runs, device=device)
    state, losses = train(Xtr, Ytr, epochs=epochs, seed=seed, device=device)
    calibrate(state, Xva, Yva)
    return state, losses, (Xva, Yva), (Xte, Yte)
