"""Seeded synthetic initial data, shared by the CUDA path and the oracle.

This module holds no arithmetic of the scheme itself (no primitive/conserved
map, no reconstruction, no flux): it only lays out primitive fields
(rho, v^x, v^y, v^z, p at cell centres) and the staggered face field
B~ = sqrt(gamma) B, built as the discrete curl of an edge-centred vector
potential so that the discrete divergence vanishes to rounding.  Each side
converts these to conserved variables with its own code.

Workloads (all seeded with ``numpy.random.default_rng(seed)``):

* ``smooth_box``: periodic special-relativistic MHD turbulence-like box in
  [0,1)^3 -- a sum of random-phase Fourier modes for rho, low-pass-filtered
  white noise for v, and a random low-k vector potential for B.  Used at 32^3
  (10 steps, the parity size), 256^3 (the throughput size) and 512^3.
* ``sweep_box``: the 256^3 variant with rho in [0.5, 1.5], log-uniform p in
  [0.1, 1], |v| <= 0.6 and B scaled so that the plasma beta spans ~1-100.
* ``linear_wave`` / ``alfven_wave``: 1-D smooth problems for convergence pins.

Host layouts: prims (5, nz, ny, nx), x fastest; face field flat, in the order
Bx (nz, ny, nx+1), By (nz, ny+1, nx), Bz (nz+1, ny, nx), face i-1/2 at index i.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

PERIODIC, OUTFLOW, AXIS = 0, 1, 2


@dataclass
class Problem:
    name: str
    n: tuple
    x0: tuple
    dx: tuple
    bc: tuple = (PERIODIC,) * 6
    metric: int = 0          # 0 flat Cartesian, 1 Kerr-Schild (ln r, theta, phi)
    spin: float = 0.0
    gamma: float = 4.0 / 3.0
    cfl: float = 0.4
    floors: bool = False
    rho_floor: float = 0.0
    rho_floor_pow: float = 0.0
    p_floor: float = 0.0
    p_floor_pow: float = 0.0
    order: int = 0           # 0 the scheme as read; 1 high order (flux-derivative correction)
    steps: int = 10
    seed: int = 0
    prims: np.ndarray = field(default=None, repr=False)   # (5, nz, ny, nx)
    bface: np.ndarray = field(default=None, repr=False)   # flat host face layout

    @property
    def ncells(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


SEED_BASE = 1810_04597


# ------------------------------------------------------------------ helpers

def _axes(n, x0, dx, off):
    """1-D coordinates of points at offset `off` (0 = centre, -0.5 = lower
    face) along each axis; face/edge arrays carry one extra point."""
    out = []
    for d in range(3):
        m = n[d] + (1 if off[d] != 0.0 else 0)
        out.append(x0[d] + (np.arange(m) + 0.5 + off[d]) * dx[d])
    return out


def _mode_sum(modes, xs):
    """sum_m a_m cos(2 pi k_m . x + phi_m) on the tensor grid xs = (x, y, z);
    returns an array (nz, ny, nx).  cos(A + B) = cos A cos B - sin A sin B
    with A along x and B on the (z, y) plane, summed over the modes as one
    matrix product."""
    x, y, z = xs
    left, right = [], []
    for (kx, ky, kz, amp, ph) in modes:
        A = 2 * np.pi * kx * x + ph
        B = 2 * np.pi * (kz * z[:, None] + ky * y[None, :])
        left += [amp * np.cos(B).reshape(-1), -amp * np.sin(B).reshape(-1)]
        right += [np.cos(A), np.sin(A)]
    acc = np.stack(left, axis=1) @ np.stack(right, axis=0)
    return acc.reshape(len(z), len(y), len(x))


def _random_k(rng, kmax):
    while True:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if np.max(np.abs(k)) >= 1:
            return k


def _random_modes(rng, count, kmax, amp_lo=0.5, amp_hi=1.0):
    modes = []
    for _ in range(count):
        k = _random_k(rng, kmax)
        modes.append((int(k[0]), int(k[1]), int(k[2]), float(rng.uniform(amp_lo, amp_hi)),
                      float(rng.uniform(0.0, 2.0 * np.pi))))
    return modes


def _lowpass_noise(rng, n, kmax, lo, hi):
    """White noise U[lo, hi] per cell, keeping only Fourier modes with
    |k|_inf <= kmax (k in units of the box): the discrete Fourier
    coefficients of those modes and their synthesis, both evaluated as
    separable sums (small matrix products) since only (2 kmax + 1)^3 modes
    survive."""
    w = rng.uniform(lo, hi, size=(n[2], n[1], n[0]))
    ks = np.arange(-kmax, kmax + 1)

    def basis(m):
        return np.exp(-2j * np.pi * np.outer(ks, np.arange(m)) / m)

    Ex, Ey, Ez = basis(n[0]), basis(n[1]), basis(n[2])
    w2 = w.reshape(-1, n[0])
    t = (w2 @ Ex.real.T + 1j * (w2 @ Ex.imag.T)).reshape(n[2], n[1], len(ks))
    t = np.einsum("zyk,jy->zjk", t, Ey)
    F = np.einsum("zjk,iz->ijk", t, Ez)                       # coefficients (kz, ky, kx)
    h = np.einsum("ijk,kx->ijx", F, Ex.conj())
    h = np.einsum("ijx,jy->iyx", h, Ey.conj()).reshape(len(ks), -1)
    Ec = Ez.conj().T
    g = Ec.real @ h.real - Ec.imag @ h.imag                   # real part of the synthesis
    return g.reshape(n[2], n[1], n[0]) / (n[0] * n[1] * n[2])


def curl_faces(n, dx, Ax, Ay, Az):
    """Face field from edge-centred vector potential components:
    Ax (nz+1, ny+1, nx) at (i, j-1/2, k-1/2), Ay (nz+1, ny, nx+1) at
    (i-1/2, j, k-1/2), Az (nz, ny+1, nx+1) at (i-1/2, j-1/2, k).
    Returns the flat host face layout (Bx, By, Bz)."""
    bx = (Az[:, 1:, :] - Az[:, :-1, :]) / dx[1] - (Ay[1:, :, :] - Ay[:-1, :, :]) / dx[2]
    by = (Ax[1:, :, :] - Ax[:-1, :, :]) / dx[2] - (Az[:, :, 1:] - Az[:, :, :-1]) / dx[0]
    bz = (Ay[:, :, 1:] - Ay[:, :, :-1]) / dx[0] - (Ax[:, 1:, :] - Ax[:, :-1, :]) / dx[1]
    return bx, by, bz


def pack_faces(bx, by, bz):
    return np.concatenate([bx.reshape(-1), by.reshape(-1), bz.reshape(-1)])


def _potential_faces(rng, n, x0, dx, kmax, count):
    """Face field of a random periodic low-k vector potential (unit scale)."""
    Ax = _mode_sum(_random_modes(rng, count, kmax), _axes(n, x0, dx, (0.0, -0.5, -0.5)))
    Ay = _mode_sum(_random_modes(rng, count, kmax), _axes(n, x0, dx, (-0.5, 0.0, -0.5)))
    Az = _mode_sum(_random_modes(rng, count, kmax), _axes(n, x0, dx, (-0.5, -0.5, 0.0)))
    return curl_faces(n, dx, Ax, Ay, Az)


def _cell_b_mag2(bx, by, bz):
    """|B|^2 from face averages (flat metric), only for scaling the seed."""
    cx = 0.5 * (bx[:, :, 1:] + bx[:, :, :-1])
    cy = 0.5 * (by[:, 1:, :] + by[:, :-1, :])
    cz = 0.5 * (bz[1:, :, :] + bz[:-1, :, :])
    return cx * cx + cy * cy + cz * cz


# ------------------------------------------------------------------ workloads

def smooth_box(n: int = 32, seed: int | None = None, steps: int = 10) -> Problem:
    """Periodic SRMHD box in [0,1)^3, Gamma = 4/3:
    rho = 1 + 0.1 * sum_{m=1..4} (1/4) cos(2 pi k_m.x + phi_m), 1 <= |k_m|_inf <= 3;
    p = 1; each v^i low-pass (|k|_inf <= 3) white noise rescaled to
    max|v^i| = 0.3; B = discrete curl of a random low-k vector potential,
    scaled so that max over faces |B~| = 0.1."""
    seed = SEED_BASE + 1 if seed is None else seed
    rng = np.random.default_rng(seed)
    nn = (n, n, n)
    x0 = (0.0, 0.0, 0.0)
    dx = (1.0 / n,) * 3
    cen = _axes(nn, x0, dx, (0.0, 0.0, 0.0))
    modes = [(int(k[0]), int(k[1]), int(k[2]), 0.25, float(rng.uniform(0, 2 * np.pi)))
             for k in (_random_k(rng, 3) for _ in range(4))]
    rho = 1.0 + 0.1 * _mode_sum(modes, cen)
    p = np.ones_like(rho)
    v = []
    for _ in range(3):
        f = _lowpass_noise(rng, nn, 3, -0.3, 0.3)
        v.append(f * (0.3 / np.max(np.abs(f))))
    bx, by, bz = _potential_faces(rng, nn, x0, dx, 3, 4)
    s = 0.1 / max(np.max(np.abs(bx)), np.max(np.abs(by)), np.max(np.abs(bz)))
    prims = np.stack([rho, v[0], v[1], v[2], p])
    return Problem(name=f"smooth_box_{n}", n=nn, x0=x0, dx=dx, steps=steps, seed=seed,
                   prims=prims, bface=pack_faces(bx * s, by * s, bz * s))


def sweep_box(n: int = 256, seed: int | None = None, steps: int = 20) -> Problem:
    """Periodic SRMHD box in [0,1)^3, Gamma = 4/3, smooth fields with
    |k|_inf <= 4: rho in [0.5, 1.5]; log10 p in [-1, 0]; |v| <= 0.6; B from a
    random vector potential scaled so that the median plasma beta
    2p/B^2 is 10 (beta then spans roughly 1-100)."""
    seed = SEED_BASE + 2 if seed is None else seed
    rng = np.random.default_rng(seed)
    nn = (n, n, n)
    x0 = (0.0, 0.0, 0.0)
    dx = (1.0 / n,) * 3
    cen = _axes(nn, x0, dx, (0.0, 0.0, 0.0))

    def unit_field():
        f = _mode_sum(_random_modes(rng, 6, 4), cen)
        return f / np.max(np.abs(f))

    rho = 1.0 + 0.5 * unit_field()
    p = 10.0 ** (-0.5 + 0.5 * unit_field())
    v = [unit_field() for _ in range(3)]
    vmag = np.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    s = 0.6 / np.max(vmag)
    v = [c * s for c in v]
    bx, by, bz = _potential_faces(rng, nn, x0, dx, 4, 6)
    b2 = _cell_b_mag2(bx, by, bz)
    beta_unit = 2.0 * p / np.maximum(b2, 1e-300)
    scale = np.sqrt(np.median(beta_unit) / 10.0)
    prims = np.stack([rho, v[0], v[1], v[2], p])
    return Problem(name=f"sweep_box_{n}", n=nn, x0=x0, dx=dx, steps=steps, seed=seed,
                   prims=prims, bface=pack_faces(bx * scale, by * scale, bz * scale))


def uniform_box(n=(8, 8, 8), rho=1.0, v=(0.2, -0.1, 0.05), p=0.7, B=(0.3, 0.2, -0.1)) -> Problem:
    """Every cell the same state (face field uniform)."""
    nn = tuple(int(x) for x in n)
    nx, ny, nz = nn
    dx = tuple(1.0 / m for m in nn)
    prims = np.empty((5, nz, ny, nx))
    prims[0] = rho
    prims[1] = v[0]
    prims[2] = v[1]
    prims[3] = v[2]
    prims[4] = p
    bx = np.full((nz, ny, nx + 1), B[0])
    by = np.full((nz, ny + 1, nx), B[1])
    bz = np.full((nz + 1, ny, nx), B[2])
    return Problem(name="uniform", n=nn, x0=(0.0, 0.0, 0.0), dx=dx, prims=prims,
                   bface=pack_faces(bx, by, bz))


def relativistic_shear(n: int = 16, speed: float = 0.99, B=(0.0, 0.0, 0.0), mirror: bool = False) -> Problem:
    """1-D periodic flow at |v| = speed whose direction turns from x to y
    over two cells in the middle (rho = p = 1, uniform face field B):
    reconstructing v^x and v^y separately gives face states with v^2 >= 1
    there.  mirror: the image under x -> -x (cells reversed, v^x negated).
    A test case for L(U) and one step: without floors the inversion fails
    within the second step (the periodic seam turns v by 90 degrees in one
    jump)."""
    ang = np.zeros(n)
    ang[n // 2:] = np.pi / 2
    ang[n // 2 - 1] = np.pi / 4
    ang[n // 2] = 3 * np.pi / 8
    prims = np.zeros((5, 1, 1, n))
    prims[0] = 1.0
    prims[4] = 1.0
    prims[1, 0, 0] = speed * np.cos(ang)
    prims[2, 0, 0] = speed * np.sin(ang)
    if mirror:
        prims = prims[..., ::-1].copy()
        prims[1] = -prims[1]
    bx = np.full((1, 1, n + 1), B[0])
    by = np.full((1, 2, n), B[1])
    bz = np.full((2, 1, n), B[2])
    return Problem(name=f"relativistic_shear_{n}", n=(n, 1, 1), x0=(0.0, 0.0, 0.0), dx=(1.0 / n, 1.0, 1.0),
                   prims=prims, bface=pack_faces(bx, by, bz))


def linear_wave(n: int, amp=0.1, v0=0.3, p0=1.0, B0=(0.2, 0.1, 0.05), t=0.0) -> Problem:
    """1-D density wave along x: rho = 1 + amp sin(2 pi (x - v0 t)), uniform
    v = (v0, 0, 0), p and B.  An exact solution of ideal (S)RMHD."""
    nn = (n, 1, 1)
    dx = (1.0 / n, 1.0, 1.0)
    x = (np.arange(n) + 0.5) / n
    prims = np.zeros((5, 1, 1, n))
    prims[0, 0, 0] = 1.0 + amp * np.sin(2 * np.pi * (x - v0 * t))
    prims[1] = v0
    prims[4] = p0
    bx = np.full((1, 1, n + 1), B0[0])
    by = np.full((1, 2, n), B0[1])
    bz = np.full((2, 1, n), B0[2])
    return Problem(name=f"linear_wave_{n}", n=nn, x0=(0.0, 0.0, 0.0), dx=dx, prims=prims,
                   bface=pack_faces(bx, by, bz))


def alfven_speed(rho=1.0, p=1.0, B0=1.0, eta=1.0, gamma=4.0 / 3.0) -> float:
    """Phase speed of the circularly polarised Alfven wave (exact nonlinear
    SRMHD solution with v^x = 0, |B_perp| = eta B0): the smaller root u of
    eta^2 B0^2 u^2 - (rho h + B0^2 (1 + eta^2)) u + B0^2 = 0, v_A = sqrt(u)."""
    rh = rho + gamma / (gamma - 1.0) * p
    bq = rh + B0 * B0 * (1.0 + eta * eta)
    u = 2.0 * B0 * B0 / (bq + np.sqrt(bq * bq - 4.0 * eta * eta * B0 ** 4))
    return float(np.sqrt(u))


def alfven_wave(n: int, t=0.0, rho=1.0, p=1.0, B0=1.0, eta=1.0, gamma=4.0 / 3.0) -> Problem:
    """Circularly polarised Alfven wave along x, phase k(x - v_A t), k = 2 pi:
    B^y = eta B0 cos, B^z = eta B0 sin, v^{y,z} = -v_A B^{y,z}/B0, v^x = 0."""
    vA = alfven_speed(rho, p, B0, eta, gamma)
    nn = (n, 1, 1)
    dx = (1.0 / n, 1.0, 1.0)
    x = (np.arange(n) + 0.5) / n
    ph = 2 * np.pi * (x - vA * t)
    By = eta * B0 * np.cos(ph)
    Bz = eta * B0 * np.sin(ph)
    prims = np.zeros((5, 1, 1, n))
    prims[0] = rho
    prims[2, 0, 0] = -vA * By / B0
    prims[3, 0, 0] = -vA * Bz / B0
    prims[4] = p
    bx = np.full((1, 1, n + 1), B0)
    by = np.stack([By, By])[:, None, :].reshape(1, 2, n)
    bz = np.stack([Bz, Bz]).reshape(2, 1, n)
    return Problem(name=f"alfven_{n}", n=nn, x0=(0.0, 0.0, 0.0), dx=dx, gamma=gamma, prims=prims,
                   bface=pack_faces(bx, by, bz))


def permute_axes(prob: Problem) -> Problem:
    """Cyclic relabelling x -> y -> z -> x of a problem (new y = old x, ...):
    the new grid's axis d+1 is the old axis d.  Returns a new Problem."""
    nx, ny, nz = prob.n
    rho, vx, vy, vz, p = prob.prims
    # arrays are (z, y, x); new axes x' = old z, y' = old x, z' = old y,
    # so the new (z', y', x') = old (y, x, z): transpose axes (1, 2, 0)
    def tr(a):
        return np.ascontiguousarray(np.transpose(a, (1, 2, 0)))
    prims = np.stack([tr(rho), tr(vz), tr(vx), tr(vy), tr(p)])
    o = 0
    bx = prob.bface[o:o + nz * ny * (nx + 1)].reshape(nz, ny, nx + 1)
    o += bx.size
    by = prob.bface[o:o + nz * (ny + 1) * nx].reshape(nz, ny + 1, nx)
    o += by.size
    bz = prob.bface[o:o + (nz + 1) * ny * nx].reshape(nz + 1, ny, nx)
    nb = (tr(bz), tr(bx), tr(by))  # new Bx' = old Bz, By' = old Bx, Bz' = old By
    n2 = (nz, nx, ny)
    dx2 = (prob.dx[2], prob.dx[0], prob.dx[1])
    x02 = (prob.x0[2], prob.x0[0], prob.x0[1])
    return Problem(name=prob.name + "_perm", n=n2, x0=x02, dx=dx2, bc=prob.bc, metric=prob.metric,
                   gamma=prob.gamma, cfl=prob.cfl, steps=prob.steps, seed=prob.seed, prims=prims,
                   bface=pack_faces(*nb))


def alfven_wave_2d(n: int, t=0.0, rho=1.0, p=1.0, B0=1.0, eta=1.0, gamma=4.0 / 3.0, order=0) -> Problem:
    """The circularly polarised Alfven wave propagating along the diagonal
    of the periodic unit square (n x n x 1), wave vector k = 2 pi (1, 1).
    order 0: the in-plane perpendicular field comes from the discrete curl of
    an edge-centred A_z, so the second-order discrete divergence vanishes;
    order 1 (for the high-order scheme): the face field holds the exact
    point values at the face centres."""
    vA = alfven_speed(rho, p, B0, eta, gamma)
    nn = (n, n, 1)
    dx = (1.0 / n, 1.0 / n, 1.0)
    kvec = np.array([2 * np.pi, 2 * np.pi])
    kmag = np.sqrt(2.0) * 2 * np.pi
    nhat = kvec / kmag
    that = np.array([-nhat[1], nhat[0]])

    def phase(x, y):
        return kvec[0] * x + kvec[1] * y - kmag * vA * t

    xc = (np.arange(n) + 0.5) / n
    xf = np.arange(n + 1) / n
    X, Y = np.meshgrid(xc, xc, indexing="xy")          # (ny, nx)
    ph = phase(X, Y)
    Bt = eta * B0 * np.cos(ph)
    Bzc = eta * B0 * np.sin(ph)
    prims = np.zeros((5, 1, n, n))
    prims[0] = rho
    vt = -vA * Bt / B0
    prims[1, 0] = vt * that[0]
    prims[2, 0] = vt * that[1]
    prims[3, 0] = -vA * Bzc / B0
    prims[4] = p
    # A_z at edges (i-1/2, j-1/2): B_perp = curl(A_z z) with
    # A_z = -(eta B0/|k|) sin(phase)
    XE, YE = np.meshgrid(xf, xf, indexing="xy")       # (ny+1, nx+1)
    Az = -(eta * B0 / kmag) * np.sin(phase(XE, YE))
    Azc = Az[None, :, :]
    if order:
        XFx, YFx = np.meshgrid(xf, xc, indexing="xy")     # x-faces (n, n+1)
        XFy, YFy = np.meshgrid(xc, xf, indexing="xy")     # y-faces (n+1, n)
        bx = (eta * B0 * np.cos(phase(XFx, YFx)) * that[0] + B0 * nhat[0])[None]
        by = (eta * B0 * np.cos(phase(XFy, YFy)) * that[1] + B0 * nhat[1])[None]
    else:
        bx = (Azc[:, 1:, :] - Azc[:, :-1, :]) / dx[1] + B0 * nhat[0]     # (1, n, n+1)
        by = -(Azc[:, :, 1:] - Azc[:, :, :-1]) / dx[0] + B0 * nhat[1]    # (1, n+1, n)
    bz = np.stack([Bzc, Bzc])                                          # (2, n, n)
    return Problem(name=f"alfven2d_{n}", n=nn, x0=(0.0, 0.0, 0.0), dx=dx, gamma=gamma, prims=prims,
                   bface=pack_faces(bx, by, bz), order=order)


# ------------------------------------------------------------------ torus

def _bl_equatorial(r, th, a):
    """Boyer-Lindquist g_tt, g_tphi, g_phiphi and Delta (M = 1)."""
    s2 = np.sin(th) ** 2
    sig = r * r + a * a * np.cos(th) ** 2
    dl = r * r - 2.0 * r + a * a
    A = (r * r + a * a) ** 2 - dl * a * a * s2
    return -(1.0 - 2.0 * r / sig), -2.0 * a * r * s2 / sig, A * s2 / sig, dl, sig, A, s2


def _fm_lnh_raw(r, th, a, ell):
    """ln(u^t) - ell * Omega for circular flow with u^t u_phi = ell.

    For u = u^t (1, 0, 0, Omega), the Euler equation of a barotropic fluid
    gives d ln h = (1/2) d g_{mn} u^m u^n = d ln u^t - ell dOmega, so
    ln h = ln u^t - ell Omega + const (Fishbone & Moncrief 1976).
    (u^t)^2 = X solves |D| X^2 - g_phiphi X - ell^2 = 0 with
    D = g_tt g_phiphi - g_tphi^2 = -Delta sin^2, and
    Omega = (ell / X - g_tphi) / g_phiphi."""
    gtt, gtp, gpp, dl, sig, A, s2 = _bl_equatorial(r, th, a)
    absD = dl * s2
    with np.errstate(divide="ignore", invalid="ignore"):
        X = (gpp + np.sqrt(gpp * gpp + 4.0 * absD * ell * ell)) / (2.0 * absD)
        om = (ell / X - gtp) / gpp
        return 0.5 * np.log(X) - ell * om, X, om


def fm_angular_momentum(a, r_max):
    """ell = u^t u_phi that puts the pressure maximum at (r_max, pi/2):
    the root of d(ln h)/dr = 0 there (found numerically)."""
    from scipy.optimize import brentq

    def dlnh(ell):
        h = 1e-5 * r_max
        return (_fm_lnh_raw(r_max + h, np.pi / 2, a, ell)[0]
                - _fm_lnh_raw(r_max - h, np.pi / 2, a, ell)[0]) / (2 * h)

    return brentq(dlnh, 1.0, 20.0, xtol=1e-14)


def ks_metric_arrays(x1, th, a):
    """Kerr-Schild lapse, shift^1 and spatial metric in (ln r, theta, phi),
    used here only to lay out the initial data (velocities, field scale)."""
    r = np.exp(x1)
    sig = r * r + a * a * np.cos(th) ** 2
    z = 2.0 * r / sig
    s2 = np.sin(th) ** 2
    alpha = 1.0 / np.sqrt(1.0 + z)
    beta1 = z / (1.0 + z) / r
    g11 = (1.0 + z) * r * r
    g13 = -a * (1.0 + z) * s2 * r
    g22 = sig
    g33 = s2 * (sig + a * a * (1.0 + z) * s2)
    return alpha, beta1, g11, g13, g22, g33


def fm_torus(n=(64, 32, 32), spin=0.9, beta=100.0, r_in=6.0, r_max=12.0, r_out=50.0, noise=0.02,
             seed=None, steps=10, with_field=True, rho_floor=1e-5, p_floor=1e-7) -> Problem:
    """Fishbone-Moncrief constant-ell torus on Kerr-Schild (ln r, theta, phi).

    Grid: ln r uniform on [ln(1.2 r_h), ln r_out], theta uniform on (0, pi),
    phi uniform on [0, 2 pi); outflow in r, polar-axis reflection in theta,
    periodic in phi.  Inside the torus (h > 1): rho = ((h - 1)/(h_max - 1))^(1/(G-1))
    (max 1), p = kappa rho^G with kappa = (h_max - 1)(G-1)/G, times (1 + noise u),
    u ~ U[-1, 1] per cell.  Velocity: the torus orbits with u^r = u^th = 0 in
    Boyer-Lindquist coordinates; those contravariant components are the same
    in Kerr-Schild, and the Eulerian 3-velocity is v^i = u^i / (alpha u^t) +
    beta^i / alpha.  Outside: atmosphere at the floors rho_floor r^-3/2,
    p_floor r^-5/2, at rest for the Eulerian observer.  Field: poloidal loops
    from A_phi = max(rho/rho_max - 0.2, 0) at the (r, theta) corners, discrete
    curl, scaled so that max p / max(b^2/2) = beta over the torus.  The
    atmosphere starts at twice the floors."""
    seed = SEED_BASE + 3 if seed is None else seed
    rng = np.random.default_rng(seed)
    gam = 4.0 / 3.0
    a = float(spin)
    nr, nt, nph = (int(v) for v in n)
    rh = 1.0 + np.sqrt(1.0 - a * a)
    x0 = (np.log(1.2 * rh), 0.0, 0.0)
    dx = ((np.log(r_out) - x0[0]) / nr, np.pi / nt, 2.0 * np.pi / nph)
    ell = fm_angular_momentum(a, r_max)
    lnh_in = _fm_lnh_raw(r_in, np.pi / 2, a, ell)[0]
    lnh_mx = _fm_lnh_raw(r_max, np.pi / 2, a, ell)[0]
    hmax = np.exp(lnh_mx - lnh_in)
    kappa = (hmax - 1.0) * (gam - 1.0) / gam

    def torus_rho(x1, th):
        r = np.exp(x1)
        lnh, X, om = _fm_lnh_raw(r, th, a, ell)
        h = np.nan_to_num(np.exp(lnh - lnh_in), nan=0.0)
        inside = (h > 1.0) & (r >= r_in)
        rho = np.where(inside, ((np.maximum(h, 1.0) - 1.0) / (hmax - 1.0)) ** (1.0 / (gam - 1.0)), 0.0)
        return rho, inside, X, om

    x1c = x0[0] + (np.arange(nr) + 0.5) * dx[0]
    thc = (np.arange(nt) + 0.5) * dx[1]
    X1, TH = np.meshgrid(x1c, thc, indexing="xy")        # (nt, nr)
    rho_t, inside, X, om = torus_rho(X1, TH)
    r = np.exp(X1)
    rho_atm = 2.0 * rho_floor * r ** -1.5     # atmosphere starts above the floors
    p_atm = 2.0 * p_floor * r ** -2.5
    alpha, beta1, g11, g13, g22, g33 = ks_metric_arrays(X1, TH, a)
    ut = np.sqrt(X)
    W = alpha * ut
    v1 = np.where(inside, beta1 / alpha, 0.0)   # u^1 = 0 in the torus
    v3 = np.where(inside, om * ut / W, 0.0)
    rho2 = np.where(inside, np.maximum(rho_t, rho_atm), rho_atm)
    p2 = np.where(inside, np.maximum(kappa * rho_t ** gam, p_atm), p_atm)
    prims = np.zeros((5, nph, nt, nr))
    prims[0] = rho2[None]
    prims[1] = v1[None]
    prims[3] = v3[None]
    pn = np.broadcast_to(p2[None], (nph, nt, nr)).copy()
    pn *= np.where(inside[None], 1.0 + noise * rng.uniform(-1.0, 1.0, size=(nph, nt, nr)), 1.0)
    prims[4] = pn

    bx = np.zeros((nph, nt, nr + 1))
    by = np.zeros((nph, nt + 1, nr))
    bz = np.zeros((nph + 1, nt, nr))
    if with_field:
        x1f = x0[0] + np.arange(nr + 1) * dx[0]
        thf = np.arange(nt + 1) * dx[1]
        XF, TF = np.meshgrid(x1f, thf, indexing="xy")   # (nt+1, nr+1) corners
        rc, _, _, _ = torus_rho(XF, TF)
        Aph = np.maximum(rc - 0.2, 0.0)
        # B~^1 = d_theta A_phi, B~^2 = -d_r A_phi (A_r = A_theta = 0)
        b1 = (Aph[1:, :] - Aph[:-1, :]) / dx[1]           # (nt, nr+1)
        b2 = -(Aph[:, 1:] - Aph[:, :-1]) / dx[0]          # (nt+1, nr)
        b2[0, :] = 0.0
        b2[-1, :] = 0.0
        # field scale from the cell-centre field (flat-index average of faces)
        sqrtg = np.sqrt((g11 * g33 - g13 * g13) * g22)
        B1 = 0.5 * (b1[:, 1:] + b1[:, :-1]) / sqrtg
        B2 = 0.5 * (b2[1:, :] + b2[:-1, :]) / sqrtg
        vl1 = g11 * v1 + g13 * v3
        vl3 = g13 * v1 + g33 * v3
        Bsq = g11 * B1 * B1 + g22 * B2 * B2
        vB = vl1 * B1
        b2c = Bsq / (W * W) + vB * vB
        pm = np.max(np.where(inside, b2c, 0.0)) / 2.0
        scale = np.sqrt(np.max(np.where(inside, p2, 0.0)) / (beta * pm)) if pm > 0 else 0.0
        bx[:] = (b1 * scale)[None]
        by[:] = (b2 * scale)[None]
        del vl3
    return Problem(name=f"fm_torus_{nr}x{nt}x{nph}", n=(nr, nt, nph), x0=x0, dx=dx,
                   bc=(OUTFLOW, OUTFLOW, AXIS, AXIS, PERIODIC, PERIODIC), metric=1, spin=a, gamma=gam,
                   floors=True, rho_floor=rho_floor, rho_floor_pow=-1.5, p_floor=p_floor, p_floor_pow=-2.5,
                   steps=steps, seed=seed, prims=prims, bface=pack_faces(bx, by, bz))


def polar_cap(n=(24, 24, 8), spin=0.9, theta_max=1.0) -> Problem:
    """A magnetised flow through the polar axis on a Kerr-Schild patch:
    ln r in [ln 4, ln 4 + 1], theta in [0, theta_max] (the axis at theta = 0,
    outflow at theta_max), phi periodic over [0, 2 pi).  Everything is smooth
    across the pole: rho = 1 + 0.1 sin^2(theta) cos(phi), p = 1, coordinate
    velocities v^1 = 0.05 cos(theta)/r, v^theta = 0.02 sin(theta) cos(theta)/r,
    v^phi = 0.01/r; the face field is the discrete coordinate curl of edge
    potentials A_phi = 0.02 sin^2(theta)/r, A_theta = 0.01 sin(theta)/r^2
    (B~^r odd in theta, B~^theta even, B~^phi odd, with div B~ = 0 to
    rounding and B~^theta = 0 on the axis faces).  No floors."""
    nr, nt, nph = (int(v) for v in n)
    x0 = (np.log(4.0), 0.0, 0.0)
    dx = (1.0 / nr, theta_max / nt, 2.0 * np.pi / nph)
    x1c, thc, phc = (x0[d] + (np.arange(n[d]) + 0.5) * dx[d] for d in range(3))
    PH, TH, X1 = np.meshgrid(phc, thc, x1c, indexing="ij")     # (nph, nt, nr)
    r = np.exp(X1)
    prims = np.zeros((5, nph, nt, nr))
    prims[0] = 1.0 + 0.1 * np.sin(TH) ** 2 * np.cos(PH)
    prims[1] = 0.05 * np.cos(TH) / r
    prims[2] = 0.02 * np.sin(TH) * np.cos(TH) / r
    prims[3] = 0.01 / r
    prims[4] = 1.0
    x1f = x0[0] + np.arange(nr + 1) * dx[0]
    thf = np.arange(nt + 1) * dx[1]
    Ax = np.zeros((nph + 1, nt + 1, nr))
    # A_theta at (i-1/2, j, k-1/2), A_phi at (i-1/2, j-1/2, k)
    Ay = np.broadcast_to((0.01 * np.sin(thc)[:, None] / np.exp(x1f)[None, :] ** 2)[None], (nph + 1, nt, nr + 1))
    Az = np.broadcast_to((0.02 * np.sin(thf)[:, None] ** 2 / np.exp(x1f)[None, :])[None], (nph, nt + 1, nr + 1))
    bx, by, bz = curl_faces((nr, nt, nph), dx, Ax, Ay, Az)
    return Problem(name=f"polar_cap_{nr}x{nt}x{nph}", n=(nr, nt, nph), x0=x0, dx=dx,
                   bc=(OUTFLOW, OUTFLOW, AXIS, OUTFLOW, PERIODIC, PERIODIC), metric=1, spin=float(spin),
                   steps=10, prims=prims, bface=pack_faces(bx, by, bz))


def michel_accretion(n_r: int, r_in=3.0, r_out=20.0, r_c=8.0, rho_c=1.0, gamma=4.0 / 3.0, order=0) -> Problem:
    """Michel (1972) steady spherical accretion of a polytropic gas (p = K
    rho^G) onto a Schwarzschild black hole (M = 1), transonic at r_c, on an
    equatorial slab of the Kerr-Schild (ln r, theta, phi) grid: n_r cells in
    ln r on [ln r_in, ln r_out], one cell in theta centred at pi/2 and one in
    phi (periodic there), outflow in r, B = 0.

    Along the radial inflow, rest-mass conservation rho u^r r^2 = C1 and the
    Bernoulli integral h^2 (1 - 2/r + (u^r)^2) = C2 hold; at the sonic
    radius (u^r)^2 = 1/(2 r_c) and c_s^2 = (u^r)^2 / (1 - 3 (u^r)^2), which
    fixes K from rho_c.  At each cell the density is the root of the
    Bernoulli relation on the subsonic branch outside r_c and the
    supersonic branch inside.  u^r is the same in Boyer-Lindquist and
    Kerr-Schild coordinates; u^t_KS = u^t_BL + (2/r)/(1 - 2/r) u^r, and the
    Eulerian velocity is v^r = u^r/(alpha u^t) + beta^r/alpha (v^x1 = v^r/r)."""
    from scipy.optimize import brentq, minimize_scalar
    G = gamma
    uc2 = 1.0 / (2.0 * r_c)
    cs2 = uc2 / (1.0 - 3.0 * uc2)
    x = cs2 / (G * (1.0 - cs2 / (G - 1.0)))          # K rho_c^(G-1)
    K = x / rho_c ** (G - 1.0)
    uc = -np.sqrt(uc2)
    h = lambda rho: 1.0 + G / (G - 1.0) * K * rho ** (G - 1.0)  # noqa: E731
    C1 = rho_c * uc * r_c * r_c
    C2 = h(rho_c) ** 2 * (1.0 - 2.0 / r_c + uc2)

    def F(lrho, r):
        rho = np.exp(lrho)
        u = C1 / (rho * r * r)
        return h(rho) ** 2 * (1.0 - 2.0 / r + u * u) - C2

    x0 = (np.log(r_in), np.pi / 2 - 0.05, 0.0)
    dx = ((np.log(r_out) - np.log(r_in)) / n_r, 0.1, 2.0 * np.pi)
    rc = np.exp(x0[0] + (np.arange(n_r) + 0.5) * dx[0])
    rho = np.empty(n_r)
    for i, r in enumerate(rc):
        lo, hi = np.log(rho_c) - 30.0, np.log(rho_c) + 30.0
        m = minimize_scalar(lambda l: F(l, r), bounds=(lo, hi), method="bounded",
                            options={"xatol": 1e-12})
        ls = m.x
        if r > r_c:
            rho[i] = np.exp(brentq(F, ls, hi, args=(r,), xtol=1e-15, rtol=1e-15))
        else:
            rho[i] = np.exp(brentq(F, lo, ls, args=(r,), xtol=1e-15, rtol=1e-15))
    u = C1 / (rho * rc * rc)
    f = 1.0 - 2.0 / rc
    ut = np.sqrt(f + u * u) / f + (2.0 / rc) / f * u
    alpha = 1.0 / np.sqrt(1.0 + 2.0 / rc)
    betar = (2.0 / rc) / (1.0 + 2.0 / rc)
    vr = u / (alpha * ut) + betar / alpha
    prims = np.zeros((5, 1, 1, n_r))
    prims[0, 0, 0] = rho
    prims[1, 0, 0] = vr / rc
    prims[4, 0, 0] = K * rho ** G
    nn = (n_r, 1, 1)
    bface = np.zeros((n_r + 1) + (1 + 1) * n_r + (1 + 1) * n_r)
    return Problem(name=f"michel_{n_r}", n=nn, x0=x0, dx=dx, bc=(OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC,
                                                                PERIODIC),
                   metric=1, spin=0.0, gamma=G, prims=prims, bface=bface, order=order)
