"""The C-ABI library builds for sm_103a, loads, exports every entry point
declared in include/echo.h, and validates configurations on the host (no
GPU needed: nothing here launches a kernel)."""
import os
import re

import pytest

from paper_1810_04597_gb300 import _lib, build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "echo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(echo_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib._SIGS, f"binding lacks {name}"


def _grid(n=(8, 8, 8), bc=(0,) * 6, dx=0.1):
    g = _lib.echo_grid()
    for d in range(3):
        g.n[d] = n[d]
        g.dx[d] = dx
    for s in range(6):
        g.bc[s] = bc[s]
    return g


def test_init_validates_and_sizes(lib):
    eos = _lib.echo_eos(4.0 / 3.0, 0, 0, 0, 0, 0)
    flat = _lib.echo_metric(0, 0.0)
    ctx = _lib.echo_init(_grid((37, 29, 23)), flat, eos, 64, 0.4)
    try:
        n = (37, 29, 23)
        N = n[0] * n[1] * n[2]
        count = 5 * N + n[2] * n[1] * (n[0] + 1) + n[2] * (n[1] + 1) * n[0] + (n[2] + 1) * n[1] * n[0]
        assert _lib.echo_state_count(ctx) == count
        padded = (n[0] + 6) * (n[1] + 6) * (n[2] + 6)
        assert _lib.echo_workspace_bytes(ctx) >= 60 * padded * 8
    finally:
        _lib.echo_destroy(ctx)
    ctx32 = _lib.echo_init(_grid((37, 29, 23)), flat, eos, 32, 0.4)
    ctx64 = _lib.echo_init(_grid((37, 29, 23)), flat, eos, 64, 0.4)
    assert _lib.echo_workspace_bytes(ctx32) < _lib.echo_workspace_bytes(ctx64)
    _lib.echo_destroy(ctx32)
    _lib.echo_destroy(ctx64)


@pytest.mark.parametrize("kw", [
    dict(n=(0, 8, 8)),
    dict(dx=-1.0),
    dict(bc=(0, 1, 0, 0, 0, 0)),
    dict(bc=(3, 3, 0, 0, 0, 0)),
])
def test_init_rejects_bad_grids(lib, kw):
    eos = _lib.echo_eos(4.0 / 3.0, 0, 0, 0, 0, 0)
    with pytest.raises(_lib.EchoError) as e:
        _lib.echo_init(_grid(**kw), _lib.echo_metric(0, 0.0), eos, 64, 0.4)
    assert e.value.code == _lib.ECHO_EINVAL


def test_init_limits_padded_arrays_to_32_bit_offsets(lib):
    """The kernels index each padded array (n + 10 per axis, x rounded up to
    8) with int offsets: echo_init takes 1278^3 (1288^3 padded < 2^31) and
    rejects 1279^3 and grids whose product would overflow."""
    eos = _lib.echo_eos(4.0 / 3.0, 0, 0, 0, 0, 0)
    flat = _lib.echo_metric(0, 0.0)
    ctx = _lib.echo_init(_grid((1278, 1278, 1278)), flat, eos, 32, 0.4)
    _lib.echo_destroy(ctx)
    for n in [(1279, 1279, 1279), (2 ** 30, 2 ** 30, 1), (1, 1, 2 ** 31 - 1), (2 ** 31 - 1, 2 ** 31 - 1, 2 ** 31 - 1)]:
        with pytest.raises(_lib.EchoError) as e:
            _lib.echo_init(_grid(n), flat, eos, 32, 0.4)
        assert e.value.code == _lib.ECHO_EINVAL, n


def test_init_rejects_bad_physics(lib):
    g = _grid()
    with pytest.raises(_lib.EchoError):
        _lib.echo_init(g, _lib.echo_metric(0, 0.0), _lib.echo_eos(1.0, 0, 0, 0, 0, 0), 64, 0.4)
    with pytest.raises(_lib.EchoError):
        _lib.echo_init(g, _lib.echo_metric(0, 0.0), _lib.echo_eos(4 / 3, 0, 0, 0, 0, 0), 16, 0.4)
    with pytest.raises(_lib.EchoError):
        _lib.echo_init(g, _lib.echo_metric(0, 0.0), _lib.echo_eos(4 / 3, 0, 0, 0, 0, 0), 64, 0.0)


def test_calls_out_of_order_are_rejected(lib):
    ctx = _lib.echo_init(_grid(), _lib.echo_metric(0, 0.0), _lib.echo_eos(4 / 3, 0, 0, 0, 0, 0), 64, 0.4)
    try:
        with pytest.raises(_lib.EchoError) as e:
            _lib.echo_step(ctx, 0.0)
        assert e.value.code == _lib.ECHO_ESTATE
        assert "echo_bind" in _lib.echo_last_error(ctx)
    finally:
        _lib.echo_destroy(ctx)


def test_totals_struct_matches_the_header(lib):
    """The binding's echo_totals has the header's members in order (the
    iteration histogram of ECHO_C2P_HIST long longs, then the counts of
    network starts and of faces the order-1 safeguard changed)."""
    import ctypes
    src = open(os.path.join(ROOT, "include", "echo.h")).read()
    body = re.search(r"typedef struct \{([^{}]*)\} echo_totals;", src).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b([a-z_0-9]+)(?:\[[A-Z_0-9]+\])?;", body)
    assert names == [f[0] for f in _lib.echo_totals._fields_], names
    assert int(re.search(r"#define ECHO_C2P_HIST (\d+)", src).group(1)) == _lib.ECHO_C2P_HIST
    assert ctypes.sizeof(_lib.echo_totals) == 8 * (7 + 6 + _lib.ECHO_C2P_HIST + 2)


def test_guess_modes_are_validated(lib):
    """Newton-start modes: 0 previous Z, 1 network, 2 cold; +4 FP32
    refinement; +8 / +16 (network on the CUDA cores / fused on the tensor
    cores) only for the network and not both.  A network mode needs a loaded
    network (ECHO_ESTATE), anything else is ECHO_EINVAL."""
    ctx = _lib.echo_init(_grid(), _lib.echo_metric(0, 0.0), _lib.echo_eos(4 / 3, 0, 0, 0, 0, 0), 64, 0.4)
    try:
        for mode in (0, 2, 4, 6):
            _lib.echo_set_c2p_guess(ctx, mode)
        for mode in (1, 5, 9, 13, 17, 21):
            with pytest.raises(_lib.EchoError) as e:
                _lib.echo_set_c2p_guess(ctx, mode)
            assert e.value.code == _lib.ECHO_ESTATE, mode
        for mode in (-1, 3, 7, 8, 10, 12, 16, 18, 25, 29, 32):
            with pytest.raises(_lib.EchoError) as e:
                _lib.echo_set_c2p_guess(ctx, mode)
            assert e.value.code == _lib.ECHO_EINVAL, mode
    finally:
        _lib.echo_destroy(ctx)


def test_kernel_names(lib):
    names = [_lib.echo_kernel_name(k) for k in range(_lib.ECHO_NK)]
    assert names[1] == "c2p" and names[3] == "faces_x" and len(set(names)) == _lib.ECHO_NK
    assert _lib.echo_kernel_name(99) == ""


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without the built library the binding raises
    instead of running anything."""
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "libecho_missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load(build_if_needed=False)


def test_static_totals_binding_checks_lengths_before_any_call():
    """echo_totals_static reads a state whose length follows from n and
    writes 6 doubles; the C entry point cannot see the buffers' lengths, so
    the binding rejects short ones before it loads or calls anything (these
    are CPU tensors: the length checks come first)."""
    import torch
    n = (4, 3, 2)
    need = _lib.static_state_count(n)
    assert need == 5 * 24 + 2 * 3 * 5 + 2 * 4 * 4 + 3 * 3 * 4
    out6 = torch.zeros(6, dtype=torch.float64)
    with pytest.raises(ValueError, match="state holds"):
        _lib.echo_totals_static(torch.zeros(need - 1, dtype=torch.float64), n, (1.0, 1.0, 1.0), out6)
    with pytest.raises(ValueError, match="out6 holds"):
        _lib.echo_totals_static(torch.zeros(need, dtype=torch.float64), n, (1.0, 1.0, 1.0),
                                torch.zeros(5, dtype=torch.float64))
    with pytest.raises(ValueError):
        _lib.echo_totals_static(torch.zeros(need, dtype=torch.float64), (4, 3), (1.0, 1.0, 1.0), out6)
    with pytest.raises(TypeError, match="device arrays"):
        _lib.echo_totals_static(torch.zeros(need, dtype=torch.float64), n, (1.0, 1.0, 1.0), out6)
