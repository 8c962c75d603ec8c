"""Pins of the oracle's high-order form (order 1): the flux-derivative
correction, the point-value MP5 interpolant and the sixth-order face-to-
centre interpolation against exact polynomial calculus; the scheme's
convergence on the oblique Alfven wave, whose fluxes are nonlinear in the
reconstructed variables (the form of order 0 is second order there); and
the conservation properties the correction must keep."""
import numpy as np
import pytest

from paper_1810_04597_gb300 import inputs


def _poly(coef, x):
    return sum(c * x ** k for k, c in enumerate(coef))


def _dpoly(coef, x):
    return sum(k * c * x ** (k - 1) for k, c in enumerate(coef) if k > 0)


def test_flux_correction_gives_exact_derivative_up_to_degree_six(orc):
    """With exact point values F(x_{j+1/2}) of a polynomial of degree <= 6,
    (Fhat_{i+1/2} - Fhat_{i-1/2}) / h equals F'(x_i) exactly; degree 7 does
    not (the correction is sixth order, not better)."""
    rng = np.random.default_rng(11)
    h = 0.37
    xs = (np.arange(-3, 3) + 0.5) * h          # interfaces x_{i-5/2} .. x_{i+5/2}, x_i = 0
    for deg in range(7):
        coef = rng.normal(size=deg + 1)
        F = _poly(coef, xs)
        lo = orc.ho_flux(F[0:5])               # Fhat at x_{i-1/2}
        hi = orc.ho_flux(F[1:6])               # Fhat at x_{i+1/2}
        assert abs((hi - lo) / h - _dpoly(coef, 0.0)) <= 1e-12 * max(1.0, np.max(np.abs(F)) / h), deg
    coef = np.zeros(8)
    coef[7] = 1.0
    F = _poly(coef, xs)
    err = abs((orc.ho_flux(F[1:6]) - orc.ho_flux(F[0:5])) / h - 0.0)
    assert err > 1e-6


def test_sixth_order_centre_interpolation_exact_up_to_degree_five(orc):
    rng = np.random.default_rng(12)
    xs = np.arange(-3, 3) + 0.5                 # faces around the centre x = 0
    for deg in range(6):
        coef = rng.normal(size=deg + 1)
        assert abs(orc.ho_center(_poly(coef, xs)) - coef[0]) <= 1e-13 * np.max(np.abs(coef)) * 100
    assert abs(orc.ho_center(xs ** 6) - 0.0) > 1e-3


def test_point_value_mp5_exact_on_quartics(orc):
    """Order 1 reconstructs point values: on a quartic sampled at the cell
    centres the unlimited interpolant equals the quartic at the interface
    (and it is the accepted value on smooth monotone data)."""
    rng = np.random.default_rng(13)
    xs = np.arange(-2, 3).astype(float)         # u_{j-2} .. u_{j+2}, interface at 0.5
    for _ in range(20):
        c = rng.normal(size=5) * np.array([1.0, 1.0, 0.1, 0.01, 0.001])
        c[1] = abs(c[1]) + 1.0                  # monotone on the stencil
        u = _poly(c, xs)
        got = orc.mp5_face_order(u, 1)
        assert abs(got - _poly(c, 0.5)) <= 1e-13 * np.max(np.abs(u)), (got, _poly(c, 0.5))
        # the cell-average interpolant (order 0) is not the point value
    u = xs ** 2
    assert abs(orc.mp5_face_order(u + 10.0 * xs, 0) - (0.25 + 5.0)) > 1e-3


def _wave_errors(orc, make, sizes, T, q, dt_of_n):
    errs = []
    for n in sizes:
        p0 = make(n, 0.0)
        ex = make(n, T)
        cfg = orc.make_cfg(p0)
        st, Z = orc.p2c(cfg, p0.prims, p0.bface)
        ns = int(np.ceil(T / dt_of_n(n)))
        st2, Z2, _, _ = orc.steps(cfg, st, Z, ns, T / ns)
        P8, _, _, _ = orc.c2p(cfg, st2, Z2)
        errs.append(np.mean(np.abs(P8[q] - ex.prims[q].reshape(-1))))
    errs = np.array(errs)
    return errs, np.log2(errs[:-1] / errs[1:])


def test_oblique_alfven_wave_high_order(orc):
    """The oblique circularly polarised Alfven wave (exact nonlinear
    solution) converges at >= 4 with the correction (order 0: second
    order).  dt ~ dx^(5/3) so that the third-order time error scales like
    dx^5."""
    make = lambda n, t: inputs.alfven_wave_2d(n, t=t, order=1)  # noqa: E731
    errs, orders = _wave_errors(orc, make, [16, 32, 64], 0.25, 3, lambda n: 0.2 / n * (16.0 / n) ** (2 / 3))
    print("oblique Alfven wave, high order: L1 errors", errs, "orders", orders)
    assert np.all(orders >= 4.0), (errs, orders)


def test_linear_wave_keeps_fifth_order(orc):
    def make(n, t):
        p = inputs.linear_wave(n, t=t)
        p.order = 1
        return p
    errs, orders = _wave_errors(orc, make, [32, 64, 128], 1.0, 0, lambda n: 0.2 / n * (32.0 / n) ** (2 / 3))
    assert np.all(orders >= 4.5), (errs, orders)


def test_high_order_conserves_and_keeps_its_divergence(orc):
    """Order 1 on the periodic parity box: mass, energy and momentum stay
    constant to rounding, and the divergence built from the corrected face
    differences (the one order 1 keeps) does not change."""
    p = inputs.smooth_box(16)
    p.order = 1
    cfg = orc.make_cfg(p)
    st, Z = orc.p2c(cfg, p.prims, p.bface)
    t0 = orc.reduce(cfg, st)
    st2, Z2, dts, stats = orc.steps(cfg, st, Z, 10)
    t1 = orc.reduce(cfg, st2)
    # reduce: mass, energy (tau), S_x, S_y, S_z, max |div B~|
    for k in (0, 1):
        assert abs(t1[k] - t0[k]) <= 1e-13 * abs(t0[k]), k
    assert np.max(np.abs(t1[2:5] - t0[2:5])) <= 1e-13 * max(1.0, np.max(np.abs(t0[2:5])))
    bmax = np.max(np.abs(st[5 * p.ncells:]))
    assert abs(t1[5] - t0[5]) * p.dx[0] <= 1e-12 * bmax, (t0[5], t1[5])


def test_high_order_state_matches_the_scheme_as_read_to_truncation(orc):
    """On a smooth box both orders approximate the same PDE: after a few
    steps the two states differ by far less than the change of the state."""
    p = inputs.smooth_box(24, seed=5)
    out = []
    for order in (0, 1):
        q = inputs.smooth_box(24, seed=5)
        q.order = order
        cfg = orc.make_cfg(q)
        st, Z = orc.p2c(cfg, q.prims, q.bface)
        st2, _, _, _ = orc.steps(cfg, st, Z, 4)
        out.append((st, st2))
    (a0, a1), (b0, b1) = out
    change = np.max(np.abs(a1 - a0))
    assert np.max(np.abs(a1 - b1)) < 0.05 * change


def test_michel_accretion_high_order(orc):
    """The same stationary Michel flow with order 1: L(U) converges at
    fifth order (D, S_r, tau; the sources use sixth-order differences of the
    metric)."""
    from test_oracle_scheme import _michel_residuals
    res, orders = _michel_residuals(orc, 1, sizes=(64, 128, 256))
    print("Michel residual orders, order 1:", orders)
    assert np.all(orders >= 4.5), (res, orders)


def _blast(n=128, contrast=1e6, B=(0.01, 0.02, 0.0)):
    """A 1-D periodic blast: a hot dense slab (rho 1, p 1) in a cold light
    medium (rho 0.1, p 1/contrast), at rest, magnetised; high-order form."""
    p = inputs.uniform_box((n, 1, 1), rho=1.0, v=(0.0, 0.0, 0.0), p=1.0, B=B)
    x = (np.arange(n) + 0.5) / n
    inside = np.abs(x - 0.5) < 0.1
    p.prims[4] = np.where(inside, 1.0, 1.0 / contrast)[None, None, :]
    p.prims[0] = np.where(inside, 1.0, 0.1)[None, None, :]
    p.order = 1
    p.dx = (1.0 / n, 1.0 / n, 1.0 / n)
    return p


@pytest.mark.parametrize("contrast", [1e4, 1e6])
def test_safeguard_keeps_a_blast_invertible(orc, contrast):
    """Pressure jumps of 1e4 and 1e6: the flux-derivative correction alone
    drives cells next to the fronts out of the invertible set; the
    safeguard returns the faces of those cells to the uncorrected flux, so
    30 steps need no floor and no failed inversion (floors are off), and
    mass and energy stay conserved to rounding on the periodic grid."""
    prob = _blast(contrast=contrast)
    cfg = orc.make_cfg(prob)
    st, Z = orc.p2c(cfg, prob.prims, prob.bface)
    t0 = orc.reduce(cfg, st)
    st1, _, _, stats = orc.steps(cfg, st, Z, 30)
    t1 = orc.reduce(cfg, st1)
    assert stats["fails"] == 0 and stats["guard_faces"] > 0, stats
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    assert abs(t1[1] - t0[1]) <= 1e-13 * abs(t0[1])


def test_safeguard_idle_on_smooth_flow(orc):
    """A smooth box: no stage result leaves the invertible set, no face is
    replaced, so the high-order form is unchanged there."""
    prob = inputs.smooth_box(16, seed=8)
    prob.order = 1
    cfg = orc.make_cfg(prob)
    st, Z = orc.p2c(cfg, prob.prims, prob.bface)
    _, _, _, stats = orc.steps(cfg, st, Z, 3)
    assert stats["guard_faces"] == 0 and stats["fails"] == 0


def test_high_order_torus_fifty_steps(orc):
    """The high-order form on the torus with its atmosphere: 50 steps stay
    finite, and the safeguard holds the inversion failures (handled by the
    floors) near the level of the scheme as read on the same grid."""
    res = {}
    for order in (0, 1):
        prob = inputs.fm_torus((40, 20, 10))
        prob.order = order
        cfg = orc.make_cfg(prob)
        st, Z = orc.p2c(cfg, prob.prims, prob.bface)
        st, Z, _, stats = orc.steps(cfg, st, Z, 50)
        assert np.all(np.isfinite(st)), order
        res[order] = stats["fails"] / stats["calls"]
    print("inversion failures per call, order 0 / order 1:", res)
    assert res[1] <= 1.25 * res[0] + 1e-3, res
