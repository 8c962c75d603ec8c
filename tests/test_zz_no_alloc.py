"""echo_totals_static: totals of a device state with no allocation.

The entry point serves callers that cannot allocate device memory when they
want these numbers (an application whose memory manager has reserved all of
HBM, a monitoring hook that must keep the device's memory footprint fixed).
Its scratch is a file-scope device array, so this test checks, through the C
ABI, that two calls in a row agree with the context-based echo_reduce.  The
file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import numpy as np
import pytest

from paper_1810_04597_gb300 import inputs

pytestmark = pytest.mark.gpu


def _totals_static(state_dev, prob, stream):
    import torch
    from paper_1810_04597_gb300 import _lib
    out = torch.full((6,), float("nan"), dtype=torch.float64, device=state_dev.device)
    _lib.echo_totals_static(state_dev, prob.n, prob.dx, out, stream.cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _agree(static, ref):
    vals = [ref["mass"], ref["energy"], *ref["mom"]]
    scale = max(abs(ref["mass"]), abs(ref["energy"]))
    for got, want in zip(static[:5], vals):
        assert abs(got - want) <= 1e-13 * scale, (got, want)
    assert abs(static[5] - ref["max_divb"]) <= 1e-13 * max(ref["max_divb"], 1e-300) + 1e-300


def test_static_totals_match_reduce_twice():
    import torch
    from paper_1810_04597_gb300.echo import Solver
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    prob = inputs.smooth_box(24, seed=31)
    s = Solver(prob)
    s.set_prims()
    state = torch.empty(s.nstate, dtype=torch.float64, device="cuda")
    for call in range(2):
        s.step()
        s.get_state(state)
        got = _totals_static(state, prob, s.stream)
        _agree(got, s.reduce())
        if call == 0:
            first = got.copy()
    assert not np.array_equal(first, got)   # second call saw the evolved state


def test_static_totals_rejects_oversized_grid():
    import torch
    from paper_1810_04597_gb300 import _lib
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.EchoError) as e:
        _lib.echo_totals_static(dummy, (4, 512, 256), (1.0, 1.0, 1.0), out)
    assert e.value.code == _lib.ECHO_ERANGE
