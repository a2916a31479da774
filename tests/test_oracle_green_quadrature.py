"""Pins of the oracle's Green's functions, hemisphere/panel rules and panel
integrals (CPU only): closed forms, symmetry, harmonicity, the reproducing
identity Eq. bw47, and library quadrature (scipy) on small cases."""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle as O
import workloads as W

A = 0.1


def _rand_in_ball(rng, n, r):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * r * rng.uniform(0, 1, (n, 1)) ** (1 / 3)


def test_green_zero_on_sphere_symmetric_and_centre_value():
    rng = np.random.default_rng(0)
    X = _rand_in_ball(rng, 50, 0.95 * A)
    S = rng.standard_normal((50, 3))
    S = A * S / np.linalg.norm(S, axis=1, keepdims=True)
    for x, s in zip(X, S):
        assert abs(O.green(A, x, s)) < 1e-12 * abs(1 / (4 * math.pi * np.linalg.norm(x - s)))
    Y = _rand_in_ball(rng, 50, 0.95 * A)
    for x, y in zip(X, Y):
        assert abs(O.green(A, x, y) - O.green(A, y, x)) < 1e-13 * abs(O.green(A, x, y))
        ry = np.linalg.norm(y)
        assert abs(O.green(A, np.zeros(3), y) - (1 / ry - 1 / A) / (4 * math.pi)) < 1e-12 / ry


def test_green_harmonic_and_gradient():
    rng = np.random.default_rng(1)
    h = 1e-4 * A
    for _ in range(10):
        x, y = _rand_in_ball(rng, 2, 0.8 * A)
        if np.linalg.norm(x - y) < 0.3 * A:
            continue
        g = O.green_grad_y(A, x, y)
        lap = -6 * O.green(A, x, y)
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            fd = (O.green(A, x, y + e) - O.green(A, x, y - e)) / (2 * h)
            assert abs(fd - g[i]) < 1e-6 * np.linalg.norm(g)
            lap += O.green(A, x, y + e) + O.green(A, x, y - e)
        assert abs(lap / h ** 2) < 1e-5 * np.linalg.norm(g) / A


def test_poisson_is_minus_normal_derivative_and_reproduces_harmonic():
    rng = np.random.default_rng(2)
    for x in _rand_in_ball(rng, 5, 0.9 * A):
        s = rng.standard_normal(3)
        y = A * s / np.linalg.norm(s)
        dn = O.green_grad_y(A, x, y) @ (y / A)
        assert abs(-dn - O.poisson(A, x, y)) < 1e-12 * abs(dn)
    # full-sphere product Gauss rule (theta in [0, pi]) of P h = h(x)
    xt, wt = O.gauss_legendre(48)
    xp, wp = O.gauss_legendre(96)
    th = 0.5 * math.pi * (xt + 1)
    ph = math.pi * (xp + 1)
    T, Ph = np.meshgrid(th, ph, indexing="ij")
    Y = A * np.stack([np.sin(T) * np.cos(Ph), np.sin(T) * np.sin(Ph), np.cos(T)], -1).reshape(-1, 3)
    Wt = (np.outer(wt * 0.5 * math.pi * np.sin(th), wp * math.pi) * A * A).reshape(-1)
    data = W.Dirichlet(W.DATA_POINT_SOURCE, x0=(0.05, 0.13, -0.02), strength=1.0)
    for x in _rand_in_ball(rng, 5, 0.6 * A):
        P = np.array([O.poisson(A, x, y) for y in Y])
        assert abs(np.sum(Wt * P) - 1.0) < 1e-10
        hv = O.dirichlet(data, Y)
        assert abs(np.sum(Wt * P * hv) - O.dirichlet(data, [x])[0]) < 1e-8


def test_hemisphere_weights_and_cap_angle():
    wl = W.cube_single_patch()
    p = O.patch_frame(wl.geometry, wl.batch.centers[0], A)
    assert p.kind == 0 and abs(p.theta_max - math.pi / 2) < 1e-15
    _, yg, Wg = O.gamma_nodes(p, 16, 16)
    assert abs(Wg.sum() - 2 * math.pi * A * A) < 1e-13
    d, _ = O.distance(wl.geometry, yg)
    assert np.all(d > 0)
    wb = W.unit_ball(n_patches=10)
    for c in wb.batch.centers:
        p = O.patch_frame(wb.geometry, c, A)
        assert abs(math.cos(p.theta_max) - A / 2) < 1e-15          # arccos(a / 2R), R = 1
        _, yg, Wg = O.gamma_nodes(p, 16, 32)
        area = 2 * math.pi * A * A * (1 - math.cos(p.theta_max))
        assert abs(Wg.sum() - area) < 1e-12 * area
        d, _ = O.distance(wb.geometry, yg)
        assert np.all(d > 0)
        # rim of the hemisphere lies on the boundary sphere
        th = p.theta_max
        Lr = A * np.array([math.sin(th), 0, -math.cos(th)])
        yr = np.array(p.c) + Lr[0] * np.array(p.t1) + Lr[2] * np.array(p.n)
        assert abs(np.linalg.norm(yr) - 1.0) < 1e-14


def test_panel_areas_and_centroids():
    wl = W.cube_single_patch()
    p = O.patch_frame(wl.geometry, wl.batch.centers[0], A)
    pan = O.panels(p, 8, 8)
    assert abs(pan["area"].sum() - math.pi * A * A) < 1e-15
    # centroid of panel 13 by library 2-D quadrature
    u0, u1, v0, v1 = pan["prm"][13][:4]
    ar = si.dblquad(lambda r, v: r, v0, v1, u0, u1, epsabs=1e-15)[0]
    cx = si.dblquad(lambda r, v: r * r * math.cos(v), v0, v1, u0, u1, epsabs=1e-15)[0] / ar
    cy = si.dblquad(lambda r, v: r * r * math.sin(v), v0, v1, u0, u1, epsabs=1e-15)[0] / ar
    assert abs(ar - pan["area"][13]) < 1e-15
    assert np.allclose(pan["Xloc"][13][:2], [cx, cy], atol=1e-13)
    # spherical cap: Archimedes, area of a cap = pi * (chord from pole to rim)^2
    wb = W.unit_ball(n_patches=3)
    p = O.patch_frame(wb.geometry, wb.batch.centers[1], A)
    pan = O.panels(p, 16, 8)
    assert abs(pan["area"].sum() - math.pi * A * A) < 1e-15
    assert np.allclose(np.linalg.norm(pan["x"], axis=1), 1.0, atol=1e-15)
    assert np.allclose(pan["normal"], pan["x"], atol=1e-14)
    d, _ = O.distance(wb.geometry, pan["x"])
    assert np.all(np.abs(d) < 1e-14)


def test_panel_integral_closed_forms_disk():
    """Flat disk through the ball centre.  Sector integral of G about the centre:
    G(0,Y) = (1/|Y| - 1/a)/4pi  =>  int_{sector r<R} = dphi (R - R^2/(2a)) / 4pi.
    Row sum from an off-centre point: the free-space part is 4 R E(rho/R) / 4pi
    (complete elliptic integral), the image part by library quadrature."""
    wl = W.cube_single_patch()
    p = O.patch_frame(wl.geometry, wl.batch.centers[0], A)
    pan = O.panels(p, 8, 8)
    dphi = 2 * math.pi / 8
    # union of the 8 inner sectors: [0, a/8] x 2pi, singular at the centre
    tot = 0.0
    for s in range(8):
        prm = pan["prm"][s].copy()
        tot += O.panel_integral(p, None, 0, np.zeros(3), prm, sing=[0.0, prm[2]])
    R = A / 8
    assert abs(tot - 2 * math.pi * (R - R * R / (2 * A)) / (4 * math.pi)) < 1e-15
    assert abs(O.panel_integral(p, None, 0, np.zeros(3), pan["prm"][3], sing=[0.0, pan["prm"][3][2]])
               - dphi * (R - R * R / (2 * A)) / (4 * math.pi)) < 1e-16
    # row sums of A from collocation points
    for i in [0, 19, 42, 63]:
        X = pan["Xloc"][i]
        rho = np.linalg.norm(X)
        row = sum(O.panel_integral(p, None, 0, X, pan["prm"][j],
                                   sing=pan["prm"][i][4:6] if i == j else None) for j in range(64))
        free = 4 * A * sp.ellipe((rho / A) ** 2) / (4 * math.pi)

        def img(r, v):
            Y = np.array([r * math.cos(v), r * math.sin(v), 0.0])
            Q = X @ X * (Y @ Y) - 2 * A * A * (X @ Y) + A ** 4
            return A / math.sqrt(Q) * r / (4 * math.pi)
        image = si.dblquad(img, 0, 2 * math.pi, 0, A, epsabs=1e-15, epsrel=1e-13)[0]
        assert abs(row - (free - image)) < 1e-12 * abs(row)


@pytest.mark.parametrize("kind", ["disk", "cap"])
def test_reproducing_identity_bw47(kind):
    """u(x) = -int_Gamma dG/dn u + int_S [-dG/dn u + G du/dn] for x inside Omega_S,
    with exact u and du/dn: pins G, grad G, P, the panel maps and Jacobians, the
    normals and the hemisphere rule without any walk."""
    if kind == "disk":
        wl = W.cube_single_patch()
        c = wl.batch.centers[0]
    else:
        wl = W.unit_ball(n_patches=50)
        c = wl.batch.centers[17]
    p = O.patch_frame(wl.geometry, c, A)
    Yl, yg, Wg = O.gamma_nodes(p, 40, 80)
    U = O.dirichlet(wl.data, yg)
    pan = O.panels(p, 4, 8)
    rng = np.random.default_rng(5)
    n, t1, t2 = np.array(p.n), np.array(p.t1), np.array(p.t2)
    for _ in range(3):
        # a point of Omega_S: inward along -n, away from S and Gamma
        L = np.array([rng.uniform(-0.2, 0.2) * A, rng.uniform(-0.2, 0.2) * A, -rng.uniform(0.3, 0.5) * A])
        xg = np.array(c) + L[0] * t1 + L[1] * t2 + L[2] * n
        dd, _ = O.distance(wl.geometry, [xg])
        assert dd[0] > 0
        gam = sum(Wg[k] * O.poisson(A, L, Yl[k]) * U[k] for k in range(len(Wg)))
        s_dl = sum(O.panel_integral(p, wl.data, 3, L, pr, rtol=1e-11) for pr in pan["prm"])
        s_sl = sum(O.panel_integral(p, wl.data, 2, L, pr, rtol=1e-11) for pr in pan["prm"])
        u = gam - s_dl + s_sl
        ue = O.dirichlet(wl.data, [xg])[0]
        assert abs(u - ue) < 1e-7 * abs(ue)


def test_flat_poisson_sum_is_half_inside():
    """For a flat S through the centre the hemisphere carries half the harmonic
    measure of the ball seen from any point of the disk (reflection symmetry)."""
    wl = W.cube_single_patch()
    p = O.patch_frame(wl.geometry, wl.batch.centers[0], A)
    pan = O.panels(p, 8, 8)
    Yl, _, Wg = O.gamma_nodes(p, 64, 128)
    for i in range(0, 40, 3):   # rings 0..4 (r < 0.63 a)
        s = sum(Wg[k] * O.poisson(A, pan["Xloc"][i], Yl[k]) for k in range(len(Wg)))
        assert abs(s - 0.5) < 2e-5
