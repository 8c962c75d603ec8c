"""Device helpers that stand in for hardware instructions, and the FP32
guess refinement of the Newton solve."""
import numpy as np
import pytest

from paper_1810_04597_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_integer_pipe_conversions_equal_hardware_casts():
    import torch
    from paper_1810_04597_gb300 import _lib
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for seed in (1, 2, 3):
        _lib.echo_selftest_conversions(1 << 22, seed, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0


def test_newton_raphson_reciprocal_within_two_ulp():
    """The c2p solve divides through a Newton-Raphson-refined reciprocal of
    the hardware's approximate one; it must stay within 2 ulp of the IEEE
    quotient."""
    import torch
    from paper_1810_04597_gb300 import _lib
    mx = torch.zeros(1, dtype=torch.int64, device="cuda")
    for seed in (4, 5):
        _lib.echo_selftest_recip(1 << 22, seed, mx)
    torch.cuda.synchronize()
    print("max ulp distance of the Newton-Raphson reciprocal:", int(mx.item()))
    assert int(mx.item()) <= 2


def test_one_step_reciprocal_within_2_pow_minus_36():
    """The c2p Newton step's quotient f / f' goes through one refinement
    step of the hardware's approximate reciprocal.  A relative error e in
    that quotient moves the converged Z by at most e tol Z (the last step
    has |dZ| <= tol Z) and leaves Newton's convergence intact for e << 1;
    with e below 2^-36 (at most 2^16 ulp of FP64) that shift is below
    1.5e-11 tol Z, far inside the FP64 parity tolerance.  Measured on GB300:
    8773 ulp (about 2^-39)."""
    import torch
    from paper_1810_04597_gb300 import _lib
    mx = torch.zeros(1, dtype=torch.int64, device="cuda")
    for seed in (4, 5):
        _lib.echo_selftest_recip1(1 << 22, seed, mx)
    torch.cuda.synchronize()
    print("max ulp distance of the one-step reciprocal:", int(mx.item()))
    assert int(mx.item()) <= 1 << 16


def test_integer_pipe_scaling_matches_fp64_products():
    """scale2 / alpha_times (exponent-field adds on the integer pipe) give
    the bit patterns of the FP64 products x*4, x*2, x*0.5 on 8 M values."""
    import torch
    from paper_1810_04597_gb300 import _lib
    bad = torch.zeros(1, dtype=torch.int64, device="cuda")
    for seed in (6, 7):
        _lib.echo_selftest_scale2(1 << 22, seed, bad)
    torch.cuda.synchronize()
    assert int(bad.item()) == 0


def test_mp5_test_from_exponents_matches_the_product():
    """The FP64 kernels decide the MP5 test a b <= eps from signs and binary
    exponents, multiplying only near eps: the same decision as the product
    test on 8 M hashed pairs (most with exponent sums at and around eps's,
    plus zeros, subnormals, huge and infinite operands)."""
    import torch
    from paper_1810_04597_gb300 import _lib
    bad = torch.zeros(1, dtype=torch.int64, device="cuda")
    for seed in (8, 9):
        _lib.echo_selftest_mp5_accept(1 << 22, seed, bad)
    torch.cuda.synchronize()
    assert int(bad.item()) == 0


@pytest.mark.parametrize("precision", [64, 32])
def test_fp32_refined_guess_converges_to_the_same_state(precision):
    """Guess mode +4 (FP32 Newton pre-refinement): same converged state as the
    plain previous-stage guess, with fewer FP64 iterations per call."""
    from paper_1810_04597_gb300.echo import Solver
    prob = inputs.sweep_box(32, seed=21)
    res = {}
    for mode in (0, 4):
        s = Solver(prob, precision=precision)
        s.set_prims()
        s.set_c2p_guess(mode)
        c0 = s.counters()
        for _ in range(3):
            s.step()
        c1 = s.counters()
        res[mode] = (s.get_state(), (c1["c2p_iters"] - c0["c2p_iters"]) / (c1["c2p_calls"] - c0["c2p_calls"]))
    a, b = res[0][0], res[4][0]
    tol = 1e-12 if precision == 64 else 1e-6
    assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(a))
    assert res[4][1] < res[0][1], (res[0][1], res[4][1])


def test_fp64_throughput_probe():
    """The FP64 FMA probe whose rate bench.py takes as the FP64 roofline
    peak: the chains stay finite and nonzero, and the measured rate lies
    between a quarter of and just above GB300's nominal FP64 peak (152 SMs x
    2 FMA x 2 flop x 2.07 GHz = 1.259 TFLOP/s): above it the launch's flop
    count would be wrong."""
    import torch
    from paper_1810_04597_gb300 import _lib
    blocks = _lib.echo_selftest_dfma_blocks()
    out = torch.empty(256 * blocks, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    _lib.echo_selftest_dfma(20000, out, s.cuda_stream)         # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    flops = _lib.echo_selftest_dfma(20000, out, s.cuda_stream)
    b.record(s)
    torch.cuda.synchronize()
    rate = flops / (a.elapsed_time(b) * 1e-3)
    print(f"FP64 FMA probe: {rate / 1e12:.3f} TFLOP/s")
    assert torch.isfinite(out).all() and (out != 0).all()
    assert 0.3e12 <= rate <= 1.05 * 1.259e12, rate
