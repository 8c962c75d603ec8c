"""Pins of the oracle's ghost fill.  Each boundary condition is one of the
padding rules of numpy.pad: periodic is 'wrap', outflow (zero gradient) is
'edge', and the polar axis is a mirror image -- 'symmetric' about the axis
for cell arrays, 'reflect' about the axis face for the face array normal to
it -- with the sign reversed for the vector component normal to the axis
and, independently, for an array that carries the factor sqrt(gamma) (odd
about the pole): the densitised face field B~ = sqrt(gamma) B is even in its
theta component and odd in the others.  Corners are filled by applying the
rule of each direction in turn (x, then y, then z), which is what the
padding of one axis after another gives."""
import numpy as np
import pytest

PERIODIC, OUTFLOW, AXIS = 0, 1, 2


def cfg_of(orc, n, bc):
    c = orc.OCfg()
    for d in range(3):
        c.n[d] = n[d]
        c.dx[d] = 1.0
    for k in range(6):
        c.bc[k] = bc[k]
    c.gamma = 4.0 / 3.0
    return c


def owned(n, g, bc_lo, d, face):
    """[lo, hi) of the owned entries along d: n cells, or the n + 1 faces of
    the d-face array (n faces when d is periodic: the last one repeats the
    first)."""
    if face == d and bc_lo != PERIODIC:
        return g, g + n + 1
    return g, g + n


def expected_fill(a, n, g, bc, comp, face, dens=0):
    out = a.copy()
    for d in range(3):
        ax = 2 - d                       # x is the fastest (last numpy) axis
        lo, hi = owned(n[d], g, bc[2 * d], d, face)
        sl = [slice(None)] * 3
        sl[ax] = slice(lo, hi)
        own = out[tuple(sl)]
        parts = []
        for side in (0, 1):
            kind = bc[2 * d + side]
            width = lo if side == 0 else a.shape[ax] - hi
            pw = [(0, 0)] * 3
            pw[ax] = (width, 0) if side == 0 else (0, width)
            if kind == AXIS:
                mode = "reflect" if face == d else "symmetric"
            else:
                mode = "wrap" if kind == PERIODIC else "edge"
            padded = np.pad(own, pw, mode=mode)
            take = [slice(None)] * 3
            take[ax] = slice(0, width) if side == 0 else slice(padded.shape[ax] - width, None)
            ghost = padded[tuple(take)]
            if kind == AXIS and ((comp == d) != bool(dens)):
                ghost = -ghost
            parts.append(ghost)
        out = np.concatenate([parts[0], own, parts[1]], axis=ax)
    return out


SETUPS = {
    "periodic": (PERIODIC,) * 6,
    "outflow": (OUTFLOW,) * 6,
    "kerr_schild": (OUTFLOW, OUTFLOW, AXIS, AXIS, PERIODIC, PERIODIC),
    "half_plane": (OUTFLOW, OUTFLOW, AXIS, OUTFLOW, PERIODIC, PERIODIC),
}


@pytest.mark.parametrize("setup", list(SETUPS))
def test_ghost_fill_is_numpy_padding(orc, setup):
    bc = SETUPS[setup]
    n = (7, 6, 8)
    g = orc.ghosts()
    cfg = cfg_of(orc, n, bc)
    rng = np.random.default_rng(40)
    shape = tuple(n[2 - k] + 2 * g for k in range(3))
    for face in (-1, 0, 1, 2):
        for comp in (-1, 0, 1, 2):
            for dens in (0, 1):
                a = np.full(shape, np.nan)
                lo = [owned(n[d], g, bc[2 * d], d, face) for d in range(3)]
                inner = (slice(*lo[2]), slice(*lo[1]), slice(*lo[0]))
                a[inner] = rng.normal(size=a[inner].shape)
                got = orc.fill_padded(cfg, a, comp, face, dens)
                want = expected_fill(a, n, g, bc, comp, face, dens)
                assert not np.isnan(got).any(), (setup, face, comp, dens)
                assert np.array_equal(got, want), (setup, face, comp, dens)


def test_axis_keeps_a_smooth_field_smooth(orc):
    """Independent of numpy: for a field smooth across the pole the polar
    (theta) component is odd and a scalar even in theta about each pole, so
    the ghost cells past both poles must hold the profile's own
    continuation: sin(2 theta) for the theta component, cos(2 theta) for a
    scalar."""
    n = (6, 12, 6)
    g = orc.ghosts()
    bc = SETUPS["kerr_schild"]
    cfg = cfg_of(orc, n, bc)
    dth = np.pi / n[1]
    th = (np.arange(n[1] + 2 * g) - g + 0.5) * dth     # cell-centre theta, ghosts beyond the poles
    shape = tuple(n[2 - k] + 2 * g for k in range(3))
    for comp, prof in ((1, np.sin(2 * th)), (-1, np.cos(2 * th))):
        a = np.full(shape, np.nan)
        inner = (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
        a[inner] = np.broadcast_to(prof[None, g:g + n[1], None], a[inner].shape)
        got = orc.fill_padded(cfg, a, comp, -1)
        col = got[g, :, g]
        # the continuation of the profile past both poles is the profile itself
        assert np.allclose(col, prof, rtol=0, atol=1e-14), comp


def test_axis_continues_the_densitised_face_field(orc):
    """Independent of numpy: the face field of an axisymmetric field smooth
    across the pole, B~^i = sqrt(gamma) B^i with sqrt(gamma) ~ sin(theta),
    continues past both poles as its own profile: B~^r ~ sin(theta) f(theta)
    with f even (odd in theta), B~^theta ~ sin(theta) sin(2 theta) (even),
    B~^phi like B~^r.  r- and phi-face arrays sit at cell-centre theta, the
    theta-face array at the faces (the axis faces hold 0)."""
    n = (6, 12, 6)
    g = orc.ghosts()
    bc = SETUPS["kerr_schild"]
    cfg = cfg_of(orc, n, bc)
    dth = np.pi / n[1]
    thc = (np.arange(n[1] + 2 * g) - g + 0.5) * dth
    thf = (np.arange(n[1] + 2 * g) - g) * dth
    shape = tuple(n[2 - k] + 2 * g for k in range(3))
    cases = ((0, np.sin(thc) * np.cos(2 * thc), n[1]), (2, np.sin(thc) * (1.0 + np.cos(thc) ** 2), n[1]),
             (1, np.sin(thf) * np.sin(2 * thf), n[1] + 1))
    for face, prof, nown in cases:
        a = np.full(shape, np.nan)
        inner = (slice(g, g + n[2]), slice(g, g + nown), slice(g, g + n[0] + (face == 0)))
        a[inner] = np.broadcast_to(prof[None, g:g + nown, None], a[inner].shape)
        got = orc.fill_padded(cfg, a, face, face, 1)
        col = got[g, :, g]
        assert np.allclose(col, prof, rtol=0, atol=1e-14), face
