"""Pins of the oracle's pointwise physics against formulations it does not use.

Every check here compares the oracle with something other than itself: the
covariant stress-energy tensor of ideal MHD built from 4-vectors, the
textbook Kerr-Schild line element, exact integrals of polynomials, the
relativistic velocity-addition law, or a finite difference.  None retypes an
oracle formula.
"""
import numpy as np
import pytest

from paper_1810_04597_gb300 import inputs

GAM = 4.0 / 3.0


def flat_cfg(orc, dx=(0.1, 0.1, 0.1)):
    p = inputs.Problem(name="pt", n=(4, 4, 4), x0=(0, 0, 0), dx=dx)
    return orc.make_cfg(p)


def ks_cfg(orc, spin=0.9, dx=(2e-3, 2e-3, 2e-3)):
    p = inputs.Problem(name="pt", n=(4, 4, 4), x0=(0, 0, 0), dx=dx, metric=1, spin=spin,
                       bc=(1, 1, 2, 2, 0, 0))
    return orc.make_cfg(p)


# ---------------------------------------------------------------- metric

def ks_line_element(x1, th, a):
    """Kerr metric in ingoing Kerr-Schild coordinates (M = 1), the standard
    line element, then x1 = ln r (dr = r dx1).  Returns g_{mu nu} 4x4."""
    r = np.exp(x1)
    sig = r * r + a * a * np.cos(th) ** 2
    s2 = np.sin(th) ** 2
    g = np.zeros((4, 4))
    g[0, 0] = -(1.0 - 2.0 * r / sig)
    g[0, 1] = g[1, 0] = 2.0 * r / sig
    g[0, 3] = g[3, 0] = -2.0 * a * r * s2 / sig
    g[1, 1] = 1.0 + 2.0 * r / sig
    g[1, 3] = g[3, 1] = -a * (1.0 + 2.0 * r / sig) * s2
    g[2, 2] = sig
    g[3, 3] = s2 * (r * r + a * a + 2.0 * a * a * r * s2 / sig)
    J = np.diag([1.0, r, 1.0, 1.0])
    return J @ g @ J


def four_metric_from_3p1(m):
    g = np.zeros((4, 4))
    bl = m["g"] @ m["beta"]
    g[0, 0] = -m["alpha"] ** 2 + bl @ m["beta"]
    g[0, 1:] = bl
    g[1:, 0] = bl
    g[1:, 1:] = m["g"]
    return g


@pytest.mark.parametrize("spin", [0.0, 0.5, 0.9, 0.98])
def test_ks_metric_matches_line_element(orc, spin):
    cfg = ks_cfg(orc, spin)
    rng = np.random.default_rng(1)
    for _ in range(50):
        x = np.array([rng.uniform(np.log(1.2), np.log(50.0)), rng.uniform(0.01, np.pi - 0.01),
                      rng.uniform(0, 2 * np.pi)])
        m = orc.metric_point(cfg, x)
        g4 = four_metric_from_3p1(m)
        ref = ks_line_element(x[0], x[1], spin)
        assert np.allclose(g4, ref, rtol=1e-14, atol=1e-14 * np.max(np.abs(ref)))
        # inverse of the spatial metric
        assert np.allclose(m["g"] @ m["gi"], np.eye(3), atol=1e-13)
        # alpha sqrt(gamma) = sqrt(-g) = r * Sigma sin(theta) in (ln r, theta, phi)
        r = np.exp(x[0])
        sig = r * r + spin * spin * np.cos(x[1]) ** 2
        assert abs(m["alpha"] * m["sqrtg"] - r * sig * np.sin(x[1])) <= 1e-13 * r * sig
        assert abs(np.sqrt(-np.linalg.det(ref)) - m["alpha"] * m["sqrtg"]) <= 1e-12 * r * sig


def test_ks_schwarzschild_limit(orc):
    cfg = ks_cfg(orc, 0.0)
    for r in [1.5, 3.0, 10.0, 40.0]:
        m = orc.metric_point(cfg, np.array([np.log(r), 1.0, 0.3]))
        assert abs(m["alpha"] - 1.0 / np.sqrt(1.0 + 2.0 / r)) < 1e-15
        # beta^r = (2/r)/(1+2/r), and beta^1 = beta^r / r in x1 = ln r
        assert abs(m["beta"][0] - (2.0 / r) / (1.0 + 2.0 / r) / r) < 1e-15


def test_flat_metric_is_identity(orc):
    m = orc.metric_point(flat_cfg(orc), np.array([0.3, 0.1, 0.7]))
    assert m["alpha"] == 1.0 and np.all(m["beta"] == 0) and np.all(m["g"] == np.eye(3))
    assert m["sqrtg"] == 1.0


# ---------------------------------------------------------------- covariant MHD

def covariant(g4, P8, gam=GAM):
    """Ideal-MHD stress-energy tensor from 4-vectors.  P8 holds the Eulerian
    3-velocity v^i and the Eulerian field B^i.  Returns conserved and flux
    vectors of the Valencia form, built only from T^{mu nu} and rho u^mu."""
    gi4 = np.linalg.inv(g4)
    alpha = 1.0 / np.sqrt(-gi4[0, 0])
    beta = alpha ** 2 * gi4[0, 1:]
    gs = g4[1:, 1:]
    rho, p = P8[0], P8[4]
    v = np.asarray(P8[1:4])
    B = np.asarray(P8[5:8])
    W = 1.0 / np.sqrt(1.0 - v @ gs @ v)
    u = np.concatenate([[W / alpha], W * (v - beta / alpha)])
    b0 = W * (v @ gs @ B) / alpha
    b = np.concatenate([[b0], (B + alpha * b0 * u[1:]) / W])
    b2 = b @ g4 @ b
    h = 1.0 + gam / (gam - 1.0) * p / rho
    T = (rho * h + b2) * np.outer(u, u) + (p + 0.5 * b2) * gi4 - np.outer(b, b)
    Tmixed = T @ g4                      # T^mu_nu
    sqrtmg = np.sqrt(-np.linalg.det(g4))
    sqrtg = np.sqrt(np.linalg.det(gs))
    cons = np.zeros(5)
    cons[0] = sqrtmg * rho * u[0]
    cons[1:4] = sqrtmg * Tmixed[0, 1:]
    cons[4] = sqrtg * alpha ** 2 * T[0, 0] - cons[0]
    flux = np.zeros((3, 5))
    for d in range(3):
        flux[d, 0] = sqrtmg * rho * u[1 + d]
        flux[d, 1:4] = sqrtmg * Tmixed[1 + d, 1:]
        flux[d, 4] = sqrtg * alpha ** 2 * T[0, 1 + d] - flux[d, 0]
    return cons, flux, T, u, b, alpha, sqrtg


def random_prims(rng, gs=None, vmax=0.9):
    """rho in [0.1,10], p/rho in [1e-2, 10], |v| <= vmax, 2p/B^2 in [0.1, 100]."""
    gs = np.eye(3) if gs is None else gs
    rho = 10 ** rng.uniform(-1, 1)
    p = rho * 10 ** rng.uniform(-2, 1)
    d = rng.normal(size=3)
    d /= np.sqrt(d @ gs @ d)
    v = d * rng.uniform(0, vmax)
    e = rng.normal(size=3)
    e /= np.sqrt(e @ gs @ e)
    beta = 10 ** rng.uniform(-1, 2)
    B = e * np.sqrt(2 * p / beta)
    return np.array([rho, v[0], v[1], v[2], p, B[0], B[1], B[2]])


def test_flux_and_conserved_match_covariant_flat(orc):
    cfg = flat_cfg(orc)
    g4 = np.diag([-1.0, 1.0, 1.0, 1.0])
    rng = np.random.default_rng(2)
    x = np.zeros(3)
    for _ in range(200):
        P = random_prims(rng)
        cons, flux, *_ = covariant(g4, P)
        C = orc.p2c_point(cfg, x, P)
        assert np.allclose(C, cons, rtol=1e-12, atol=1e-13 * np.max(np.abs(cons)))
        for d in range(3):
            F, U = orc.flux_point(cfg, x, P, d)
            scale = np.max(np.abs(flux[d])) + np.max(np.abs(cons))
            assert np.allclose(F, flux[d], atol=1e-13 * scale)
            assert np.allclose(U, cons, atol=1e-13 * scale)


@pytest.mark.parametrize("spin", [0.0, 0.9])
def test_flux_and_conserved_match_covariant_ks(orc, spin):
    cfg = ks_cfg(orc, spin)
    rng = np.random.default_rng(3)
    for _ in range(100):
        x = np.array([rng.uniform(np.log(1.5), np.log(40.0)), rng.uniform(0.2, np.pi - 0.2),
                      rng.uniform(0, 2 * np.pi)])
        g4 = ks_line_element(x[0], x[1], spin)
        P = random_prims(rng, g4[1:, 1:], vmax=0.8)
        cons, flux, *_ = covariant(g4, P)
        m = orc.metric_point(cfg, x)
        C = orc.p2c_point(cfg, x, P) * m["sqrtg"]
        scale_c = np.max(np.abs(cons))
        assert np.allclose(C, cons, atol=1e-12 * scale_c)
        for d in range(3):
            F, U = orc.flux_point(cfg, x, P, d)
            scale = np.max(np.abs(flux[d])) + scale_c
            assert np.allclose(F, flux[d], atol=1e-12 * scale), (d, F, flux[d])


# ---------------------------------------------------------------- c2p

@pytest.mark.parametrize("metric", ["flat", "ks"])
def test_c2p_roundtrip(orc, metric):
    """c2p(p2c(P)) = P to 1e-13 on rho in [0.1,10], p/rho in [1e-2,10],
    |v| <= 0.9, 2p/B^2 in [0.1,100], from the cold guess."""
    rng = np.random.default_rng(4)
    cfg = flat_cfg(orc) if metric == "flat" else ks_cfg(orc, 0.9)
    worst = 0.0
    for _ in range(2000):
        if metric == "flat":
            x = np.zeros(3)
            gs = np.eye(3)
        else:
            x = np.array([rng.uniform(np.log(1.5), np.log(40.0)), rng.uniform(0.2, np.pi - 0.2), 1.0])
            gs = orc.metric_point(cfg, x)["g"]
        P = random_prims(rng, gs)
        C = orc.p2c_point(cfg, x, P)
        rc, P5, Z, it = orc.c2p_point(cfg, x, C, P[5:8], 0.0)
        assert rc == 0
        vmag = np.sqrt(P[1:4] @ gs @ P[1:4])
        err = max(abs(P5[0] - P[0]) / P[0], abs(P5[4] - P[4]) / P[4],
                  np.max(np.abs(P5[1:4] - P[1:4])) / max(vmag, 1e-3))
        worst = max(worst, err)
    assert worst <= 1e-13, worst


def test_c2p_stress_domain(orc):
    """Wider domain (magnetisation up to 1e3, |v| up to 0.99): the error
    grows with W and sigma; recorded, with a loose bound."""
    rng = np.random.default_rng(5)
    cfg = flat_cfg(orc)
    worst = 0.0
    for _ in range(500):
        rho = 10 ** rng.uniform(-1, 1)
        p = rho * 10 ** rng.uniform(-2, 1)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        v = d * rng.uniform(0.9, 0.99)
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        sigma = 10 ** rng.uniform(0, 3)
        B = e * np.sqrt(sigma * rho)
        P = np.array([rho, *v, p, *B])
        C = orc.p2c_point(cfg, np.zeros(3), P)
        rc, P5, Z, it = orc.c2p_point(cfg, np.zeros(3), C, B, 0.0)
        assert rc == 0
        worst = max(worst, abs(P5[4] - p) / p, abs(P5[0] - rho) / rho)
    assert worst < 1e-7, worst


def test_c2p_residual_vanishes_at_exact_Z(orc):
    """f(Z*) = 0 at Z* = rho h W^2 of the primitives: the residual is the
    energy definition rewritten in Z."""
    rng = np.random.default_rng(6)
    cfg = flat_cfg(orc)
    for _ in range(300):
        P = random_prims(rng)
        C = orc.p2c_point(cfg, np.zeros(3), P)
        rho, p = P[0], P[4]
        W2 = 1.0 / (1.0 - P[1:4] @ P[1:4])
        Zs = (rho + GAM / (GAM - 1) * p) * W2
        f, fp = orc.c2p_residual(cfg, np.zeros(3), C, P[5:8], Zs)
        assert abs(f) <= 1e-13 * (C[4] + C[0])


def test_c2p_derivative_matches_finite_difference(orc):
    rng = np.random.default_rng(7)
    cfg = flat_cfg(orc)
    for _ in range(300):
        P = random_prims(rng)
        C = orc.p2c_point(cfg, np.zeros(3), P)
        W2 = 1.0 / (1.0 - P[1:4] @ P[1:4])
        Z = (P[0] + 4 * P[4]) * W2 * rng.uniform(1.0, 1.5)
        h = 1e-5 * Z
        fa, _ = orc.c2p_residual(cfg, np.zeros(3), C, P[5:8], Z + h)
        fb, _ = orc.c2p_residual(cfg, np.zeros(3), C, P[5:8], Z - h)
        _, fp = orc.c2p_residual(cfg, np.zeros(3), C, P[5:8], Z)
        assert abs((fa - fb) / (2 * h) - fp) <= 1e-7 * max(1.0, abs(fp))


def test_c2p_converges_quadratically_from_previous_guess(orc):
    """A guess within 1% converges in at most 4 iterations."""
    rng = np.random.default_rng(8)
    cfg = flat_cfg(orc)
    for _ in range(200):
        P = random_prims(rng, vmax=0.6)
        C = orc.p2c_point(cfg, np.zeros(3), P)
        W2 = 1.0 / (1.0 - P[1:4] @ P[1:4])
        Zs = (P[0] + 4 * P[4]) * W2
        rc, P5, Z, it = orc.c2p_point(cfg, np.zeros(3), C, P[5:8], Zs * (1 + 0.01 * rng.uniform(-1, 1)))
        assert rc == 0 and it <= 4


# ---------------------------------------------------------------- speeds / HLL

def test_speeds_velocity_addition_sound(orc):
    """B = 0, v along d: lambda = (v +- c_s)/(1 +- v c_s), c_s^2 = G p/(rho h)."""
    cfg = flat_cfg(orc)
    for rho, p, v in [(1.0, 1.0, 0.3), (0.2, 5.0, -0.7), (3.0, 0.01, 0.95)]:
        cs = np.sqrt(GAM * p / (rho + GAM / (GAM - 1) * p))
        for d in range(3):
            P = np.zeros(8)
            P[0], P[4] = rho, p
            P[1 + d] = v
            lp, lm = orc.speeds_point(cfg, np.zeros(3), P, d)
            assert abs(lp - (v + cs) / (1 + v * cs)) < 1e-14
            assert abs(lm - (v - cs) / (1 - v * cs)) < 1e-14


def test_speeds_perpendicular_fast_wave(orc):
    """Field transverse to d, v along d: in the fluid frame the wave vector is
    perpendicular to the field, where the relativistic fast magnetosonic speed
    is exact, a^2 = (G p + b^2)/(rho h + b^2) (total-enthalpy form of the
    RMHD dispersion relation; b^2 = B^2/W^2 since v.B = 0), and the lab speeds
    follow by velocity addition along d."""
    cfg = flat_cfg(orc)
    for rho, p, v, bmag in [(1.0, 0.5, 0.0, 0.8), (0.3, 2.0, 0.6, 1.5), (2.0, 0.05, -0.9, 0.4)]:
        W2 = 1.0 / (1.0 - v * v)
        b2 = bmag * bmag / W2
        a = np.sqrt((GAM * p + b2) / (rho + GAM / (GAM - 1) * p + b2))
        for d in range(3):
            P = np.zeros(8)
            P[0], P[4] = rho, p
            P[1 + d] = v
            P[5 + (d + 1) % 3] = bmag
            lp, lm = orc.speeds_point(cfg, np.zeros(3), P, d)
            assert abs(lp - (v + a) / (1 + v * a)) < 1e-14
            assert abs(lm - (v - a) / (1 - v * a)) < 1e-14


def test_speeds_cold_alfven_limit(orc):
    """p -> 0 with v = 0: a -> the relativistic Alfven speed
    B^2/(rho + B^2) (comoving field at rest)."""
    cfg = flat_cfg(orc)
    P = np.array([1.0, 0, 0, 0, 1e-300, 0.3, 0.4, 0.0])
    lp, lm = orc.speeds_point(cfg, np.zeros(3), P, 0)
    ca = np.sqrt(0.25 / 1.25)
    assert abs(lp - ca) < 1e-14 and abs(lm + ca) < 1e-14


def test_speeds_at_rest_in_ks(orc):
    """v = 0: lambda = +- alpha a sqrt(gamma^dd) - beta^d."""
    cfg = ks_cfg(orc, 0.9)
    x = np.array([np.log(5.0), 1.1, 0.0])
    m = orc.metric_point(cfg, x)
    P = np.array([1.0, 0, 0, 0, 0.5, 0, 0, 0])
    cs = np.sqrt(GAM * 0.5 / (1 + 4 * 0.5))
    for d in range(3):
        lp, lm = orc.speeds_point(cfg, x, P, d)
        ref = m["alpha"] * cs * np.sqrt(m["gi"][d, d])
        assert abs(lp - (ref - m["beta"][d])) < 1e-14
        assert abs(lm - (-ref - m["beta"][d])) < 1e-14


def test_hll_identical_states_and_static_pressure(orc):
    cfg = flat_cfg(orc)
    rng = np.random.default_rng(9)
    P = random_prims(rng)
    F, U = orc.flux_point(cfg, np.zeros(3), P, 1)
    lp, lm = orc.speeds_point(cfg, np.zeros(3), P, 1)
    Fh = orc.hll(F, F, U, U, max(0, lp), max(0, -lm))
    assert np.allclose(Fh, F, rtol=1e-15, atol=1e-15)
    # static unmagnetised state: momentum flux = p delta, others zero
    P = np.array([2.0, 0, 0, 0, 0.7, 0, 0, 0])
    for d in range(3):
        F, U = orc.flux_point(cfg, np.zeros(3), P, d)
        ref = np.zeros(5)
        ref[1 + d] = 0.7
        assert np.array_equal(F, ref)


def test_hll_supersonic_picks_upwind(orc):
    """All waves moving right: a- = 0, F_HLL = F_L."""
    cfg = flat_cfg(orc)
    PL = np.array([1.0, 0.9, 0, 0, 0.1, 0, 0, 0])
    PR = np.array([0.5, 0.9, 0.1, 0, 0.2, 0, 0, 0])
    FL, UL = orc.flux_point(cfg, np.zeros(3), PL, 0)
    FR, UR = orc.flux_point(cfg, np.zeros(3), PR, 0)
    lpL, lmL = orc.speeds_point(cfg, np.zeros(3), PL, 0)
    lpR, lmR = orc.speeds_point(cfg, np.zeros(3), PR, 0)
    am = max(0.0, -lmL, -lmR)
    assert am == 0.0
    F = orc.hll(FL, FR, UL, UR, max(0.0, lpL, lpR), am)
    assert np.allclose(F, FL, rtol=1e-15, atol=1e-15)


# ---------------------------------------------------------------- MP5

def cell_averages(coef, x0, h, count):
    """Exact averages of the polynomial sum_k coef[k] x^k over cells
    [x0 + j h, x0 + (j+1) h]."""
    P = np.polynomial.Polynomial(coef)
    I = P.integ()
    edges = x0 + h * np.arange(count + 1)
    return (I(edges[1:]) - I(edges[:-1])) / h, P


def test_mp5_unlimited_exact_on_quartic_averages(orc):
    """The unlimited MP5 value is the fifth-order interpolant of cell
    averages: exact at the interface for polynomials of degree <= 4."""
    rng = np.random.default_rng(10)
    for _ in range(200):
        coef = rng.normal(size=5)
        h = rng.uniform(0.05, 0.5)
        avg, P = cell_averages(coef, -2.5 * h, h, 5)
        val = orc.mp5_unlimited(avg)
        assert abs(val - P(0.5 * h)) <= 1e-12 * max(1.0, np.max(np.abs(avg)))
    # and not exact for degree 5
    avg, P = cell_averages([0, 0, 0, 0, 0, 1.0], -2.5, 1.0, 5)
    assert abs(orc.mp5_unlimited(avg) - P(0.5)) > 1e-6


def test_mp5_limiter_inactive_on_smooth_monotone(orc):
    rng = np.random.default_rng(11)
    for _ in range(500):
        a = rng.uniform(0.5, 2.0)
        h = rng.uniform(0.01, 0.1)
        x = rng.uniform(-1, 1) + h * np.arange(-2, 3)
        u = np.exp(a * x)
        assert orc.mp5_face(u) == orc.mp5_unlimited(u)


def test_mp5_step_has_no_overshoot(orc):
    """At a jump the limited value is the upwind value (no new extremum)."""
    assert orc.mp5_face([0, 0, 0, 1, 1]) == 0.0
    assert orc.mp5_face([0, 0, 1, 1, 1]) == 1.0
    assert orc.mp5_face([1, 1, 1, 0, 0]) == 1.0
    assert orc.mp5_face([2, 2, 2, 2, 2]) == pytest.approx(2.0, abs=1e-15)
    rng = np.random.default_rng(12)
    for _ in range(2000):
        u = np.sort(rng.uniform(-1, 1, size=5))
        if rng.uniform() < 0.5:
            u = u[::-1]
        val = orc.mp5_face(u)
        assert min(u[2], u[3]) - 1e-15 <= val <= max(u[2], u[3]) + 1e-15


# ---------------------------------------------------------------- sources

def christoffel0(g4fun, x, h):
    """Gamma^0_{mu nu} of a stationary metric by fourth-order differences."""
    g4 = g4fun(x)
    gi4 = np.linalg.inv(g4)
    dg = np.zeros((4, 4, 4))   # dg[l] = d_l g_{mu nu}
    for d in range(3):
        acc = np.zeros((4, 4))
        for w, o in [(1, -2), (-8, -1), (8, 1), (-1, 2)]:
            y = x.copy()
            y[d] += o * h
            acc += w * g4fun(y)
        dg[1 + d] = acc / (12 * h)
    G0 = np.zeros((4, 4))
    for mu in range(4):
        for nu in range(4):
            G0[mu, nu] = 0.5 * sum(gi4[0, l] * (dg[mu][l, nu] + dg[nu][l, mu] - dg[l][mu, nu])
                                   for l in range(4))
    return G0, dg


@pytest.mark.parametrize("spin", [0.0, 0.9])
def test_sources_match_covariant_form(orc, spin):
    """sqrt(gamma) S(S_j) = 1/2 sqrt(-g) T^{mu nu} d_j g_{mu nu};
    sqrt(gamma) S(tau) = sqrt(-g) (T^{mu 0} d_mu alpha - alpha T^{mu nu} Gamma^0_{mu nu})."""
    h = 2e-3
    cfg = ks_cfg(orc, spin, dx=(h, h, h))
    rng = np.random.default_rng(13)

    def g4fun(y):
        return ks_line_element(y[0], y[1], spin)

    for _ in range(30):
        x = np.array([rng.uniform(np.log(2.0), np.log(30.0)), rng.uniform(0.3, np.pi - 0.3), 0.4])
        g4 = g4fun(x)
        P = random_prims(rng, g4[1:, 1:], vmax=0.7)
        cons, flux, T, u, b, alpha, sqrtg = covariant(g4, P)
        G0, dg = christoffel0(g4fun, x, h)
        sqrtmg = np.sqrt(-np.linalg.det(g4))
        ref = np.zeros(5)
        for j in range(3):
            ref[1 + j] = 0.5 * sqrtmg * np.sum(T * dg[1 + j])
        # d_mu alpha, alpha = (-g^00)^(-1/2)
        dal = np.zeros(4)
        for d in range(3):
            acc = 0.0
            for w, o in [(1, -2), (-8, -1), (8, 1), (-1, 2)]:
                y = x.copy()
                y[d] += o * h
                acc += w / np.sqrt(-np.linalg.inv(g4fun(y))[0, 0])
            dal[1 + d] = acc / (12 * h)
        ref[4] = sqrtmg * (T[:, 0] @ dal - alpha * np.sum(T * G0))
        src = orc.sources_point(cfg, x, P)
        scale = np.max(np.abs(ref)) + 1e-300
        assert np.allclose(src, ref, atol=1e-8 * scale, rtol=0), (src, ref)


def test_sources_vanish_in_flat_space(orc):
    cfg = flat_cfg(orc)
    P = random_prims(np.random.default_rng(14))
    assert np.all(orc.sources_point(cfg, np.zeros(3), P) == 0.0)
