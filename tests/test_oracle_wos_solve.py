"""Pins of the oracle's walk-on-spheres, LU, patch solve and potential (CPU only):
mean-value property, exact harmonic solutions within 4 SE + epsilon shell bias,
a library solver, closed-form Neumann data, and the representation formula."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def test_walk_absorbs_inside_shell_and_caps():
    g = W.Geometry(W.GEOM_BALL_INTERIOR, radius=1.0)
    d = W.Dirichlet(W.DATA_CONSTANT, constant=2.5)
    o = O.wos_opts(eps=1e-3)
    ok, sc, st = O.walk(g, d, np.array([0.9995, 0, 0]), 0, 0, 0, o)
    assert ok and st == 1 and sc == 2.5
    o = O.wos_opts(eps=1e-3, max_steps=1)
    ok, sc, st = O.walk(g, d, np.array([0.2, 0, 0]), 0, 0, 0, o)
    assert not ok and st == 1


@pytest.mark.parametrize("stream", [O.STREAM_F64, O.STREAM_F32])
def test_first_jump_uniform_on_sphere(stream):
    """From the ball centre the first sphere is the boundary itself, so every
    walk is absorbed after one jump at a uniform point of the unit sphere;
    scoring Y_lm (l = 1, 2) gives mean 0 within 4 SE (mean-value property)."""
    g = W.Geometry(W.GEOM_BALL_INTERIOR, radius=1.0)
    o = O.wos_opts(eps=1e-9, stream=stream)
    N = 40000
    for l, m in [(1, -1), (1, 0), (1, 1), (2, -2), (2, 0), (2, 1)]:
        c = np.zeros(9)
        c[l * l + l + m] = 1.0
        d = W.Dirichlet(W.DATA_HARMONIC_SH, lmax=2, clm=c)
        res = O.wos_points(g, d, np.zeros((1, 3)), [l * 10 + m + 5], [3], [N], o)
        U, SE = O.wos_estimates(res, N)
        assert int(res["steps"][0]) == 2 * N
        assert abs(U[0]) < 4 * SE[0]


def test_martingale_diagnostic_unbiased():
    """Scoring the harmonic data at the absorption point itself (not at its
    projection) is exactly unbiased: E u(x_tau) = u(y)."""
    wl = W.unit_ball(n_patches=4)
    o = O.wos_opts(eps=1e-2, score=1)
    y = np.array([[0.3, -0.2, 0.5], [0.0, 0.9, 0.1], [-0.6, 0.1, -0.2]])
    N = 20000
    res = O.wos_points(wl.geometry, wl.data, y, [0, 1, 2], [0], [N], o)
    U, SE = O.wos_estimates(res, N)
    ue = O.dirichlet(wl.data, y)
    assert np.all(np.abs(U - ue) < 4 * SE)


@pytest.mark.parametrize("which", ["cube_point_source", "ball_harmonic", "wires"])
def test_wos_vs_exact_within_4se_plus_shell(which):
    if which == "cube_point_source":
        wl = W.cube_single_patch()
        y = W.points_in_box(12, (0.3, 0.3, 0.0), (0.7, 0.7, 0.2), margin=0.0)
    elif which == "ball_harmonic":
        wl = W.unit_ball(n_patches=4)
        y = W.targets_in_ball(12, 1.0, 0.05)
    else:
        boxes = np.array([[0.3, 0.3, 0.3, 0.6, 0.5, 0.45], [0.1, 0.6, 0.6, 0.9, 0.8, 0.7]])
        geom = W.Geometry(W.GEOM_BOX_MINUS_BOXES, lo=(0, 0, 0), hi=(1, 1, 1), boxes=boxes)
        data = W.Dirichlet(W.DATA_POINT_SOURCE, x0=(0.45, 0.4, 0.375))
        wl = W.Workload("wires_small", geom, data, None)
        y = W.points_in_box(40, (0.05, 0.05, 0.05), (0.95, 0.95, 0.95), margin=0.0)
        inside = np.zeros(len(y), bool)
        for b in boxes:
            inside |= np.all((y > b[:3] - 0.05) & (y < b[3:] + 0.05), axis=1)
        y = y[~inside][:12]
    N = 8000
    eps = 1e-4
    res = O.wos_points(wl.geometry, wl.data, y, np.arange(len(y)), [9], [N], O.wos_opts(eps=eps))
    U, SE = O.wos_estimates(res, N)
    ue = O.dirichlet(wl.data, y)
    # shell bias: at most eps * sup |grad u| on the shell
    if which == "ball_harmonic":
        L = 50.0 * np.sum(np.abs(wl.data.clm))
    else:
        dmin = 0.3 if which == "cube_point_source" else 0.05
        L = 1.0 / (4 * math.pi * dmin ** 2)
    assert np.all(np.abs(U - ue) <= 4 * SE + eps * L)
    assert np.all(res["capped"] == 0)


def test_lu_vs_library():
    rng = np.random.default_rng(0)
    for n in [1, 5, 64, 129]:
        A = rng.standard_normal((n, n)) + n * 0.1 * np.eye(n)
        b = rng.standard_normal(n)
        x = O.lu_solve(A, b)
        assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-11, atol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        O.lu_solve(np.zeros((3, 3)), np.ones(3))


def _rel_inner(q, qe, Xloc, a):
    m = np.linalg.norm(Xloc, axis=1) < 0.7 * a
    return np.linalg.norm((q - qe)[m]) / np.linalg.norm(qe[m])


def test_patch_solve_exact_u_disk_closed_form():
    """C1 geometry with exact u at the nodes: q vs the point-source Neumann data
    0.3 / (4 pi |x - x0|^3); piecewise-constant collocation gives ~1% inside
    r < 0.7a (the paper reports < 1.25% there, Sec. 5.2)."""
    wl = W.cube_single_patch()
    c = wl.batch.centers[0]
    p = O.patch_frame(wl.geometry, c, 0.1)
    _, yg, _ = O.gamma_nodes(p, 16, 16)
    U = O.dirichlet(wl.data, yg)
    r = O.solve_patch(wl.geometry, wl.data, c, 0.1, 16, 16, 8, 8, 0, 0, O.wos_opts(), U_in=U)
    pan = O.panels(p, 8, 8)
    d = pan["x"] - np.array([0.5, 0.5, -0.3])
    qe = 0.3 / (4 * math.pi * np.linalg.norm(d, axis=1) ** 3)
    assert np.allclose(O.neumann_exact(wl.data, pan["x"], pan["normal"]), qe, rtol=1e-13)
    assert _rel_inner(r["q"], qe, pan["Xloc"], 0.1) < 0.02
    # finer hemisphere rule: smaller error (discretisation, not a bug)
    _, yg2, _ = O.gamma_nodes(p, 32, 64)
    r2 = O.solve_patch(wl.geometry, wl.data, c, 0.1, 32, 64, 8, 8, 0, 0, O.wos_opts(),
                       U_in=O.dirichlet(wl.data, yg2))
    assert _rel_inner(r2["q"], qe, pan["Xloc"], 0.1) < 0.5 * _rel_inner(r["q"], qe, pan["Xloc"], 0.1)


def test_patch_solve_exact_u_cap_closed_form():
    wl = W.unit_ball(n_patches=20)
    c = wl.batch.centers[5]
    p = O.patch_frame(wl.geometry, c, 0.1)
    _, yg, _ = O.gamma_nodes(p, 16, 32)
    U = O.dirichlet(wl.data, yg)
    r = O.solve_patch(wl.geometry, wl.data, c, 0.1, 16, 32, 8, 8, 0, 5, O.wos_opts(), U_in=U,
                      rtol=1e-10)
    pan = O.panels(p, 8, 8)
    qe = np.array([sum(l * wl.data.clm[l * l + l + m] * O.real_sh(8, x)[l * l + l + m]
                       for l in range(9) for m in range(-l, l + 1)) for x in pan["x"]])
    assert _rel_inner(r["q"], qe, pan["Xloc"], 0.1) < 0.04


def test_constant_data_gives_zero_neumann():
    wl = W.unit_ball(n_patches=20)
    d = W.Dirichlet(W.DATA_CONSTANT, constant=3.0)
    c = wl.batch.centers[2]
    p = O.patch_frame(wl.geometry, c, 0.1)
    r = O.solve_patch(wl.geometry, d, c, 0.1, 8, 16, 4, 8, 0, 0, O.wos_opts(),
                      U_in=np.full(128, 3.0), rtol=1e-10)
    assert np.max(np.abs(r["q"])) < 1e-10


def test_full_patch_with_walks_small():
    """Steps 1 and 2 together with walks; q(WOS) stays within a few percent of
    q(exact U) at a small walk count."""
    wl = W.cube_single_patch()
    c = wl.batch.centers[0]
    o = O.wos_opts(eps=1e-4)
    r = O.solve_patch(wl.geometry, wl.data, c, 0.1, 8, 8, 4, 8, 2000, 0, o, rtol=1e-10)
    p = O.patch_frame(wl.geometry, c, 0.1)
    _, yg, _ = O.gamma_nodes(p, 8, 8)
    ue = O.dirichlet(wl.data, yg)
    assert np.all(np.abs(r["U"] - ue) < 4 * r["SE"] + 1e-4 * 1.0)
    rx = O.solve_patch(wl.geometry, wl.data, c, 0.1, 8, 8, 4, 8, 0, 0, o, U_in=ue, rtol=1e-10)
    assert np.linalg.norm(r["q"] - rx["q"]) / np.linalg.norm(rx["q"]) < 0.1
    assert r["steps"] > 8 * 8 * 2000


def test_representation_formula_inside_and_outside():
    """Eq. bw03 with exact Dirichlet/Neumann data on a panel cover of the unit
    sphere (Voronoi-owned panels of Fibonacci patches): u inside, 0 outside."""
    wl = W.unit_ball(n_patches=300, a=0.25)
    xs, ns, ar, own = [], [], [], []
    for i, c in enumerate(wl.batch.centers):
        p = O.patch_frame(wl.geometry, c, 0.25)
        pan = O.panels(p, 12, 16)
        xs.append(pan["x"]); ns.append(pan["normal"]); ar.append(pan["area"])
        own.append(np.full(len(pan["area"]), i))
    xs, ns, ar, own = map(np.concatenate, (xs, ns, ar, own))
    keep = O.owned(xs, own, wl.batch.centers)
    xs, ns, ar = xs[keep], ns[keep], ar[keep]
    assert abs(ar.sum() - 4 * math.pi) < 0.04 * 4 * math.pi
    g = O.dirichlet(wl.data, xs)
    q = O.neumann_exact(wl.data, xs, ns)
    tin = W.targets_in_ball(6, 1.0, 0.4)
    tout = W.targets_outside_ball(6, 1.0, 0.4)
    uin = O.potential(xs, ns, ar, q, g, tin)
    uout = O.potential(xs, ns, ar, q, g, tout)
    ue = O.dirichlet(wl.data, tin)
    scale = np.max(np.abs(g))
    assert np.max(np.abs(uin - ue)) < 0.02 * scale
    assert np.max(np.abs(uout)) < 0.02 * scale
