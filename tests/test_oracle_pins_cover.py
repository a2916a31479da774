"""Pins of the oracle parts that set tolerances or decide ownership elsewhere:
the jump direction of a walk (Sec. 2), the majorants of the representation sum
Eq. bw03 that scale every fast-multipole tolerance, and the Voronoi ownership
of the overlapping patch cover (Sec. 6, lowest index on ties).  Each is checked
against what the mathematics fixes, not against its own formula."""
import math

import numpy as np
import pytest

import oracle as O


# ------------------------------------------------------------ jump direction
@pytest.mark.parametrize("stream", [O.STREAM_F64, O.STREAM_F32])
def test_direction_unit_and_quadrant_points(stream):
    """z = 1 - 2 u1 and a full turn of azimuth: known points of the sphere."""
    # u1 = 1/2: the equator; u1 = 1/4: z = 1/2
    for u1, z in [(0.5, 0.0), (0.25, 0.5), (0.75, -0.5)]:
        for u2 in np.linspace(0.01, 0.99, 7):
            om = O.direction(u1, u2, stream)
            assert abs(np.linalg.norm(om) - 1.0) < 1e-15
            assert om[2] == z
    # the azimuth at u2 = 1/4, 1/2, 3/4 on the equator: stream 0 turns 2 pi u2,
    # stream 1 turns 2 pi (u2 - 1/2)
    want = {O.STREAM_F64: {0.25: [0, 1, 0], 0.5: [-1, 0, 0], 0.75: [0, -1, 0]},
            O.STREAM_F32: {0.25: [0, -1, 0], 0.5: [1, 0, 0], 0.75: [0, 1, 0]}}[stream]
    for u2, v in want.items():
        assert np.allclose(O.direction(0.5, u2, stream), v, atol=1e-15)


@pytest.mark.parametrize("stream", [O.STREAM_F64, O.STREAM_F32])
def test_direction_is_isotropic(stream):
    """The first and second moments of a uniform direction on the sphere are 0
    and I/3; a midpoint grid of uniforms reproduces them to O(h^2)."""
    n = 120
    u = (np.arange(n) + 0.5) / n
    om = np.array([O.direction(a, b, stream) for a in u for b in u])
    assert np.max(np.abs(om.mean(axis=0))) < 1e-12
    M = om.T @ om / len(om)
    assert np.max(np.abs(M - np.eye(3) / 3.0)) < 1e-4


def test_streams_differ_by_half_turn_only():
    """Stream 1 turns the azimuth of stream 0 by pi about z (reading R3): the
    same uniform law, x and y negated, z kept."""
    rng = np.random.default_rng(5)
    for u1, u2 in rng.random((40, 2)):
        a = O.direction(u1, u2, O.STREAM_F64)
        b = O.direction(u1, u2, O.STREAM_F32)
        assert np.allclose(b, [-a[0], -a[1], a[2]], atol=1e-14)


# ------------------------------------------------------- potential majorants
def _cloud(seed, n, nt):
    rng = np.random.default_rng(seed)
    y = rng.normal(size=(n, 3))
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    area = rng.uniform(0.01, 0.1, n)
    q = rng.normal(size=n)
    g = rng.normal(size=n)
    t = rng.normal(size=(nt, 3)) * 2.0
    return y, nrm, area, q, g, t


def test_majorants_equal_independent_sums():
    """b0 = sum |A q| / (4 pi r) and b1 = sum |A g| / (4 pi r^2), summed here with
    NumPy from the definition (a dropped 4 pi or a wrong power of r fails)."""
    y, nrm, area, q, g, t = _cloud(1, 300, 40)
    b0, b1 = O.potential_majorants(y, area, q, g, t)
    r = np.linalg.norm(t[:, None, :] - y[None, :, :], axis=2)
    e0 = (np.abs(area * q)[None, :] / (4 * math.pi * r)).sum(axis=1)
    e1 = (np.abs(area * g)[None, :] / (4 * math.pi * r ** 2)).sum(axis=1)
    assert np.allclose(b0, e0, rtol=1e-13, atol=0)
    assert np.allclose(b1, e1, rtol=1e-13, atol=0)


def test_majorants_bound_each_layer_and_are_sharp():
    """|single layer| <= b0 and |double layer| <= b1 per target; both become
    equalities for one panel whose normal points at the target."""
    y, nrm, area, q, g, t = _cloud(2, 200, 30)
    b0, b1 = O.potential_majorants(y, area, q, g, t)
    single = O.potential(y, nrm, area, q, np.zeros_like(g), t)
    double = O.potential(y, nrm, area, np.zeros_like(q), g, t)
    assert np.all(np.abs(single) <= b0 * (1 + 1e-14))
    assert np.all(np.abs(double) <= b1 * (1 + 1e-14))
    # one panel at the origin, normal towards the target: |u| reaches the bound
    t1 = np.array([[0.3, -0.4, 1.2]])
    n1 = -t1 / np.linalg.norm(t1)   # (t - y).n = -|t - y|: the dipole term is +|A g|/(4 pi r^2)
    y1, a1, q1, g1 = np.zeros((1, 3)), np.array([0.07]), np.array([-2.5]), np.array([1.75])
    c0, c1 = O.potential_majorants(y1, a1, q1, g1, t1)
    s = O.potential(y1, n1, a1, q1, np.zeros(1), t1)
    d = O.potential(y1, n1, a1, np.zeros(1), g1, t1)
    assert abs(abs(s[0]) - c0[0]) <= 1e-15 * c0[0]
    assert abs(abs(d[0]) - c1[0]) <= 1e-15 * c1[0]


# --------------------------------------------------------- Voronoi ownership
def test_owned_lowest_index_wins_exact_ties():
    """A point equidistant (exactly, in FP64) from several centres belongs to
    the lowest index among them."""
    cen = np.array([[2.0, 0.0, 0.0], [-2.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 3.0]])
    x = np.zeros((1, 3))
    # centres 0, 1, 2 are at distance 2, centre 3 at 3: owner 0 keeps, 1 and 2 do not
    assert O.owned(x, [0], cen).tolist() == [True]
    assert O.owned(x, [1], cen).tolist() == [False]
    assert O.owned(x, [2], cen).tolist() == [False]
    # reorder: the same point now belongs to whichever tied centre comes first
    cen2 = cen[[3, 2, 1, 0]]
    assert O.owned(x, [1], cen2).tolist() == [True]
    assert O.owned(x, [2], cen2).tolist() == [False]
    assert O.owned(x, [3], cen2).tolist() == [False]


def test_owned_matches_brute_force_argmin():
    """Random panels and centres, with duplicated centres (exact ties): keep[i]
    iff owner[i] is the first index of the minimum squared distance (NumPy's
    argmin takes the first index on ties)."""
    rng = np.random.default_rng(7)
    cen = rng.integers(-4, 5, size=(30, 3)).astype(float)
    cen = np.concatenate([cen, cen[:10]])   # exact duplicates at indices 30..39
    x = rng.integers(-8, 9, size=(2000, 3)).astype(float) * 0.5   # many exact ties
    d2 = ((x[:, None, :] - cen[None, :, :]) ** 2).sum(axis=2)
    best = np.argmin(d2, axis=1)
    own = rng.integers(0, len(cen), size=len(x))
    own[::3] = best[::3]
    dup = best < 10
    own[np.where(dup)[0][::2]] = best[np.where(dup)[0][::2]] + 30   # the duplicate must lose
    keep = O.owned(x, own, cen)
    assert np.array_equal(keep, own == best)
    assert keep.sum() > 500 and (~keep).sum() > 500
