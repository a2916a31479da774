"""Pins of the oracle's RNG, Gauss rules, geometry and data functions (CPU only).

Each test checks the oracle against something other than itself: published
known-answer vectors, a library routine, a closed form, brute force or an
invariant the mathematics fixes.
"""
import math
import os

import numpy as np
import pytest
import scipy.special as sp

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    assert list(O.philox(ctr, key)) == out


def test_uniform_conversions_open_interval_and_grid():
    assert O.u01_21(0) == 2.0 ** -22
    assert O.u01_21(0x1FFFFF) == 1.0 - 2.0 ** -22
    assert O.u01_53(0, 0) == 2.0 ** -53
    assert O.u01_53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    rng = np.random.default_rng(1)
    for f in rng.integers(0, 2 ** 21, 200):
        u = O.u01_21(int(f))
        k = u * 2 ** 22
        assert 0.0 < u < 1.0 and k == int(k) and int(k) == 2 * int(f) + 1


def test_fields21_use_every_bit_once():
    """The six 21-bit fields of a Philox block are disjoint: together they take
    126 of its 128 bits, all but bit 10 of words 1 and 3."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        w = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        f = O.fields21(w)
        assert np.all(f < 2 ** 21)
        assert [int(v) for v in f[:4]] == [int(x) >> 11 for x in w]
        assert int(f[4]) == (int(w[0]) & 0x7FF) | ((int(w[1]) & 0x3FF) << 11)
        assert int(f[5]) == (int(w[2]) & 0x7FF) | ((int(w[3]) & 0x3FF) << 11)
    # flipping any bit outside bit 10 of words 1 and 3 changes exactly one field
    w = np.zeros(4, dtype=np.uint32)
    base = O.fields21(w)
    for i in range(4):
        for b in range(32):
            v = w.copy()
            v[i] = np.uint32(1 << b)
            changed = int(np.sum(O.fields21(v) != base))
            assert changed == (0 if (i in (1, 3) and b == 10) else 1), (i, b)
    # the uniforms built from Philox words are uniform: KS test on 20000 draws
    us = [O.u01_53(*O.philox([i, 7, 3, 1], [0, 0])[:2]) for i in range(20000)]
    from scipy.stats import kstest
    assert kstest(us, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("n", [1, 2, 5, 10, 16, 32, 64])
def test_gauss_legendre_vs_library(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 1e-14
    assert np.max(np.abs(w - wr)) < 1e-14
    # exact for degree 2n-1
    for d in range(2 * n):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) < 1e-13


def _surface_samples_box(lo, hi, n, rng):
    lo, hi = np.asarray(lo), np.asarray(hi)
    pts = rng.uniform(lo, hi, size=(n, 3))
    f = rng.integers(0, 6, n)
    ax, side = f // 2, f % 2
    pts[np.arange(n), ax] = np.where(side == 0, lo[ax], hi[ax])
    return pts


def test_distance_ball_invariants():
    g = W.Geometry(W.GEOM_BALL_INTERIOR, center=(0.1, -0.2, 0.3), radius=1.5)
    rng = np.random.default_rng(0)
    x = np.array(g.center) + rng.uniform(-1, 1, (200, 3)) * 0.8
    d, nb = O.distance(g, x)
    assert np.allclose(np.linalg.norm(nb - np.array(g.center), axis=1), 1.5, atol=1e-14)
    assert np.allclose(np.linalg.norm(x - nb, axis=1), d, atol=1e-13)
    # brute force over points of the sphere
    v = rng.standard_normal((20000, 3))
    s = np.array(g.center) + 1.5 * v / np.linalg.norm(v, axis=1, keepdims=True)
    bf = np.min(np.linalg.norm(x[:, None, :] - s[None], axis=2), axis=1)
    assert np.all(d <= bf + 1e-12) and np.all(bf - d < 0.05)


def test_distance_box_and_wires_brute_force():
    rng = np.random.default_rng(2)
    boxes = np.array([[0.2, 0.2, 0.2, 0.4, 0.5, 0.3], [0.6, 0.1, 0.5, 0.9, 0.3, 0.8]])
    for g in [W.Geometry(W.GEOM_BOX_INTERIOR, lo=(0, 0, 0), hi=(1, 2, 1)),
              W.Geometry(W.GEOM_BOX_MINUS_BOXES, lo=(0, 0, 0), hi=(1, 1, 1), boxes=boxes)]:
        # random interior points (outside obstacles)
        x = rng.uniform(g.lo, g.hi, size=(400, 3))
        if g.boxes is not None:
            inside = np.zeros(len(x), bool)
            for b in boxes:
                inside |= np.all((x > b[:3]) & (x < b[3:]), axis=1)
            x = x[~inside]
        d, nb = O.distance(g, x)
        assert np.allclose(np.linalg.norm(x - nb, axis=1), d, atol=1e-14)
        s = [_surface_samples_box(g.lo, g.hi, 60000, rng)]
        if g.boxes is not None:
            for b in boxes:
                s.append(_surface_samples_box(b[:3], b[3:], 20000, rng))
        s = np.concatenate(s)
        bf = np.min(np.linalg.norm(x[:, None, :] - s[None], axis=2), axis=1)
        assert np.all(d <= bf + 1e-12)
        assert np.all(bf - d < 0.03)


def test_real_sh_vs_scipy():
    rng = np.random.default_rng(3)
    lmax = 8
    for _ in range(20):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        th = math.acos(v[2])
        ph = math.atan2(v[1], v[0])
        Y = O.real_sh(lmax, v)
        for l in range(lmax + 1):
            for m in range(-l, l + 1):
                c = sp.sph_harm_y(l, abs(m), th, ph)   # complex, Condon-Shortley phase included
                cs = (-1) ** abs(m)
                if m == 0:
                    ref = c.real
                elif m > 0:
                    ref = math.sqrt(2) * cs * c.real
                else:
                    ref = math.sqrt(2) * cs * c.imag
                assert abs(Y[l * l + l + m] - ref) < 1e-12


def test_sh_data_harmonic_and_neumann_closed_form():
    """r^l Y_lm is harmonic (finite-difference Laplacian); on the unit sphere the
    radial derivative of sum c_lm r^l Y_lm is sum l c_lm Y_lm."""
    wl = W.unit_ball(n_patches=4)
    d = wl.data
    rng = np.random.default_rng(4)
    h = 1e-3
    for _ in range(5):
        x = rng.uniform(-0.5, 0.5, 3)
        lap = -6 * O.dirichlet(d, x)[0]
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            lap += O.dirichlet(d, x + e)[0] + O.dirichlet(d, x - e)[0]
        assert abs(lap / h ** 2) < 1e-4 * np.sum(np.abs(d.clm)) * 10
    pts = W.fibonacci_sphere(30)
    qn = O.neumann_exact(d, pts, pts)
    for x, q in zip(pts, qn):
        Y = O.real_sh(8, x)
        ref = sum(l * d.clm[l * l + l + m] * Y[l * l + l + m] for l in range(9) for m in range(-l, l + 1))
        assert abs(q - ref) < 1e-10 * max(1.0, abs(ref))


def test_point_source_neumann_matches_paper_test1():
    with open(os.path.join(GOLDEN, "paper_test1_neumann.txt")) as f:
        row = [float(t) for t in f.read().split("\n")[-2].split()]
    x, x0, n, val = row[0:3], row[3:6], row[6:9], row[9]
    d = W.Dirichlet(W.DATA_POINT_SOURCE, x0=tuple(x0), strength=4 * math.pi)
    q = O.neumann_exact(d, [x], [n])[0]
    assert abs(q - val) < 5e-6
