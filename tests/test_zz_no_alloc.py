"""echo_totals_static: totals of a device state with no allocation.

The entry point serves callers that cannot allocate device memory when they
want these numbers (an application whose memory manager has reserved all of
HBM, a monitoring hook that must keep the device's memory footprint fixed).
Its scratch is a file-scope device array, so this test checks, through the C
ABI, that two calls in a row agree with the context-based echo_reduce and
that a call changes neither torch's allocated bytes nor the device's free
bytes.  The
file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest

from paper_1810_04597_gb300 import inputs

pytestmark = pytest.mark.gpu


def _totals_static(state_dev, prob, stream, out):
    import torch
    from paper_1810_04597_gb300 import _lib
    out.fill_(float("nan"))
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
    from paper_1810_04597_gb300 import _lib
    from paper_1810_04597_gb300.echo import Solver
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    prob = inputs.smooth_box(24, seed=31)
    s = Solver(prob)
    s.set_prims()
    state = torch.empty(s.nstate, dtype=torch.float64, device="cuda")
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    nn = (ctypes.c_int * 3)(*prob.n)
    dd = (ctypes.c_double * 3)(*prob.dx)
    for call in range(2):
        s.step()
        s.get_state(state)
        if call == 1:
            # the defining property: a call allocates no device memory, neither
            # through torch's allocator nor behind it (free bytes of the device)
            torch.cuda.synchronize()
            alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
            rc = _lib.load().echo_totals_static(ctypes.c_void_p(state.data_ptr()), nn, dd,
                                                ctypes.c_void_p(out.data_ptr()),
                                                ctypes.c_void_p(s.stream.cuda_stream))
            assert rc == _lib.ECHO_OK
            torch.cuda.synchronize()
            assert torch.cuda.memory_allocated() == alloc0
            assert torch.cuda.mem_get_info()[0] == free0
        got = _totals_static(state, prob, s.stream, out)
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
    nn = (ctypes.c_int * 3)(4, 512, 256)
    dd = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    # through the C ABI: the row count is checked before any pointer is used
    rc = _lib.load().echo_totals_static(ctypes.c_void_p(dummy.data_ptr()), nn, dd,
                                        ctypes.c_void_p(out.data_ptr()), None)
    assert rc == _lib.ECHO_ERANGE


def test_static_totals_rejects_host_pointers():
    import torch
    from paper_1810_04597_gb300 import _lib
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    prob = inputs.smooth_box(8, seed=3)
    n_state = _lib.static_state_count(prob.n)
    host_state = np.zeros(n_state)
    dev_state = torch.zeros(n_state, dtype=torch.float64, device="cuda")
    host_out = np.zeros(6)
    dev_out = torch.zeros(6, dtype=torch.float64, device="cuda")
    nn = (ctypes.c_int * 3)(*prob.n)
    dd = (ctypes.c_double * 3)(*prob.dx)
    fn = _lib.load().echo_totals_static
    # pageable host memory for either pointer: rejected, nothing launched
    assert fn(ctypes.c_void_p(host_state.ctypes.data), nn, dd, ctypes.c_void_p(dev_out.data_ptr()),
              None) == _lib.ECHO_EINVAL
    assert fn(ctypes.c_void_p(dev_state.data_ptr()), nn, dd, ctypes.c_void_p(host_out.ctypes.data),
              None) == _lib.ECHO_EINVAL
    torch.cuda.synchronize()
    assert float(dev_out.abs().sum()) == 0.0
