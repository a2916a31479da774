"""Oracle pins for wrapped patches on the wire layout (a ball about a point of an
obstacle face that meets further faces of the same box, reading R15): the face
pieces of S and their areas (closed forms of disk segments and brute force),
the hemisphere Gamma (its area in closed form for an edge patch, the
star-shaped test), the panel maps (areas and normals), and the reproducing
identity Eq. bw47 with exact data, which pins G, dG/dn, the Poisson kernel,
the pieces' Jacobians and normals together."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

A = 0.3
BOX = np.array([1.0, 1.0, 1.0, 3.0, 1.8, 1.7])   # one wire 2 x 0.8 x 0.7 in a 4 x 3 x 3 box


def _geo(box=BOX):
    return W.Geometry(W.GEOM_BOX_MINUS_BOXES, lo=(0, 0, 0), hi=(4, 3, 3), boxes=np.array([box]))


def _data():
    # a point source inside the wire: harmonic in the region, exact Neumann data known
    return W.Dirichlet(W.DATA_POINT_SOURCE, x0=(2.0, 1.4, 1.35), strength=1.0)


def test_edge_patch_pieces_and_areas_closed_form():
    """Centre on the top face at distance d = 0.1 from its long edge: S is the
    top disk of radius a less the segment beyond the edge, a^2 acos(d/a) -
    d sqrt(a^2 - d^2), plus a half disk of radius sqrt(a^2 - d^2) on the side
    face.  The pieces' panels (several ring and sector counts) add up to these
    areas and carry the two faces' normals (into the box)."""
    d = 0.1
    p = O.patch_frame(_geo(), (2.0, 1.0 + d, 1.7), A)
    assert p.kind == 2 and p.npiece == 2
    seg = A * A * math.acos(d / A) - d * math.sqrt(A * A - d * d)
    top = math.pi * A * A - seg
    side = 0.5 * math.pi * (A * A - d * d)
    areas = [pc[2] for pc in p.pieces()]
    assert abs(areas[0] - top) < 1e-13 and abs(areas[1] - side) < 1e-13
    for nr, ns in ((2, 8), (4, 24), (7, 13)):
        pan = O.panels(p, nr, ns)
        assert abs(pan["area"].sum() - (top + side)) < 1e-12
        normals = {tuple(np.round(v, 12)) for v in pan["normal"]}
        assert normals == {(0.0, 0.0, -1.0), (0.0, 1.0, 0.0)}
        # every collocation point lies on the box surface and inside the ball
        x = pan["x"]
        assert np.all(np.linalg.norm(x - np.array([2.0, 1.1, 1.7]), axis=1) < A)
        on_top = np.isclose(x[:, 2], 1.7, rtol=0, atol=1e-15) & (x[:, 1] >= 1.0)
        on_side = np.isclose(x[:, 1], 1.0, rtol=0, atol=1e-15) & (x[:, 2] <= 1.7)
        assert np.all(on_top | on_side)


def test_corner_patch_area_brute_force():
    """Centre near a corner of the top face: three pieces; their areas agree with
    a fine grid count of the box surface inside the ball."""
    c = np.array([3.0 - 0.12, 1.8 - 0.15, 1.7])
    p = O.patch_frame(_geo(), c, A)
    assert p.kind == 2 and p.npiece == 3
    lo, hi = BOX[:3], BOX[3:]
    tot, h = 0.0, 1e-4
    for ax in range(3):
        for side in range(2):
            fv = hi[ax] if side else lo[ax]
            o = [i for i in range(3) if i != ax]
            us = np.arange(max(lo[o[0]], c[o[0]] - A) + h / 2, min(hi[o[0]], c[o[0]] + A), h)
            vs = np.arange(max(lo[o[1]], c[o[1]] - A) + h / 2, min(hi[o[1]], c[o[1]] + A), h)
            U, V = np.meshgrid(us, vs, indexing="ij")
            tot += np.count_nonzero((U - c[o[0]]) ** 2 + (V - c[o[1]]) ** 2 + (fv - c[ax]) ** 2 < A * A) * h * h
    assert abs(sum(pc[2] for pc in p.pieces()) - tot) < 2e-6


def test_edge_patch_gamma_area_closed_form():
    """Gamma = the sphere outside the box.  For the edge patch the sphere inside
    the box is {z <= 0} cut by {y >= -d}: by the mirror symmetry in z it is half
    the zone {y >= -d}, of area 2 pi a (a + d), so |Gamma| = pi a (3a - d).  The
    product rule of theta_max(phi) (Gauss in phi over the full turn) converges
    to it, slowly: theta_max has square-root kinks in phi."""
    d = 0.1
    p = O.patch_frame(_geo(), (2.0, 1.0 + d, 1.7), A)
    exact = math.pi * A * (3 * A - d)
    errs = []
    for nph in (64, 256, 1024):
        _, _, Wg = O.gamma_nodes(p, 16, nph)
        errs.append(abs(Wg.sum() - exact) / exact)
    assert errs[0] < 5e-3 and errs[1] < 1e-4 and errs[2] < 2e-5
    assert errs[2] < errs[1] < errs[0]
    # every node lies in the region, on the sphere
    _, yg, _ = O.gamma_nodes(p, 16, 64)
    assert np.allclose(np.linalg.norm(yg - np.array([2.0, 1.1, 1.7]), axis=1), A, rtol=0, atol=1e-15)
    dd, _ = O.distance(_geo(), yg)
    assert np.all(dd >= -1e-15)


def test_thin_wire_is_not_star_shaped_and_other_conductors_rejected():
    """A wire thinner than a: the arc from the pole passes through the wire and
    comes out behind it, so Gamma is not star-shaped about the pole; a ball
    reaching a second conductor is rejected too."""
    thin = np.array([1.0, 1.0, 1.0, 3.0, 1.8, 1.2])   # 0.2 thick
    with pytest.raises(ValueError):
        O.patch_frame(_geo(thin), (2.0, 1.4, 1.2), A)
    two = W.Geometry(W.GEOM_BOX_MINUS_BOXES, lo=(0, 0, 0), hi=(4, 3, 3),
                     boxes=np.array([BOX, [1.0, 2.0, 1.0, 3.0, 2.5, 1.7]]))
    with pytest.raises(ValueError):
        O.patch_frame(two, (2.0, 1.8 - 0.05, 1.5), A)   # side face; the ball reaches the second wire
    with pytest.raises(ValueError):
        O.patch_frame(_geo(), (2.0, 1.0, 1.2), 1.1)     # the ball reaches the outer box


@pytest.mark.parametrize("where", ["edge", "corner"])
def test_reproducing_identity_bw47_wrapped(where):
    """u(x) = sum_k W_k P(x, y_k) u(y_k) - int_S dG/dn_y u + int_S G du/dn for x
    in Omega_S = B cap D, with the exact point-source data: to the accuracy
    of the Gamma rule (1024 azimuths)."""
    c = {"edge": (2.0, 1.1, 1.7), "corner": (3.0 - 0.12, 1.8 - 0.15, 1.7)}[where]
    geo, data = _geo(), _data()
    p = O.patch_frame(geo, c, A)
    assert p.kind == 2
    Yl, yg, Wg = O.gamma_nodes(p, 24, 1024)
    U = O.dirichlet(data, yg)
    pan = O.panels(p, 3, 16)
    n, t1, t2 = np.array(p.n), np.array(p.t1), np.array(p.t2)
    rng = np.random.default_rng(3)
    for _ in range(3):
        # a point of Omega_S above the face, away from S and Gamma
        L = np.array([rng.uniform(-0.25, 0.25) * A, rng.uniform(-0.25, 0.25) * A, -rng.uniform(0.3, 0.6) * A])
        xg = np.array(c) + L[0] * t1 + L[1] * t2 + L[2] * n
        dd, _ = O.distance(geo, [xg])
        assert dd[0] > 0.05
        gam = sum(Wg[k] * O.poisson(A, L, Yl[k]) * U[k] for k in range(len(Wg)))
        s_dl = sum(O.panel_integral(p, data, 3, L, pr, rtol=1e-11) for pr in pan["prm"])
        s_sl = sum(O.panel_integral(p, data, 2, L, pr, rtol=1e-11) for pr in pan["prm"])
        ue = O.dirichlet(data, [xg])[0]
        assert abs(gam - s_dl + s_sl - ue) < 1e-4 * abs(ue)


def test_wrapped_solve_with_exact_values_away_from_edges():
    """The collocation solve with the exact u at the hemisphere nodes: panels
    away from the box edges (the Neumann data are singular at a re-entrant
    edge) within 3% of the exact Neumann data; the panel counts of a wrapped
    patch are rings x sectors."""
    geo, data = _geo(), _data()
    c = (2.0, 1.1, 1.7)
    p = O.patch_frame(geo, c, A)
    nt, nph, nr, ns = 16, 64, 4, 24
    _, yg, _ = O.gamma_nodes(p, nt, nph)
    r = O.solve_patch(geo, data, c, A, nt, nph, nr, ns, 0, 0, O.wos_opts(), U_in=O.dirichlet(data, yg), rtol=1e-10)
    pan = O.panels(p, nr, ns)
    assert r["q"].shape == (nr * ns,)
    qe = O.neumann_exact(data, pan["x"], pan["normal"])
    x = pan["x"]
    dist_edge = np.minimum(np.abs(x[:, 1] - 1.0) + np.abs(x[:, 2] - 1.7), 1.0)
    far = dist_edge > 0.08
    assert far.sum() >= 20
    err = np.abs(r["q"] - qe)[far] / np.max(np.abs(qe[far]))
    assert np.max(err) < 0.03, np.max(err)


def test_right_side_converged_with_a_distant_source():
    """The right side's data integrals are refined relative to their own size:
    with the source of the wire workload 30 units away (g(y) - g(x) ~ 1e-4 of
    the kernel's scale) the right side at rtol 1e-10 agrees with rtol 1e-12 to
    1e-11 of max|b| (with the tolerance taken from the size of G alone they
    differed by 1e-8)."""
    wl = W.wires(n_patches=16, walks=2)
    b = wl.batch
    p = int(np.nonzero(wl.faces_met == 3)[0][0])
    pf = O.patch_frame(wl.geometry, b.centers[p], float(b.radius[p]))
    nt, nph, nr, ns = int(b.n_theta[p]), int(b.n_phi[p]), int(b.n_rings[p]), int(b.n_sectors[p])
    _, yg, _ = O.gamma_nodes(pf, nt, nph)
    U = O.dirichlet(wl.data, yg)
    _, b10 = O.assemble(pf, wl.data, nr, ns, nt, nph, U, rtol=1e-10)
    _, b12 = O.assemble(pf, wl.data, nr, ns, nt, nph, U, rtol=1e-12)
    assert np.max(np.abs(b10 - b12)) <= 1e-11 * np.max(np.abs(b12))


def test_polar_origin_moves_onto_a_near_side():
    """A centre 0.002 from the long edge of the top face: the top piece's polar
    origin moves onto that edge (0.002 < rf/4); left where it was, the rings of
    the strip between it and the edge would be panels 0.6 long and 0.0005 wide.
    The pieces keep their closed-form areas and the collocation matrix stays
    well conditioned."""
    d = 0.002
    geo, data = _geo(), _data()
    p = O.patch_frame(geo, (2.0, 1.0 + d, 1.7), A)
    q = p.piece[0]
    assert q.ax == 2 and q.onlo[1] == 1 and q.P[1] == 1.0 and q.P[0] == 2.0
    seg = A * A * math.acos(d / A) - d * math.sqrt(A * A - d * d)
    areas = [pc[2] for pc in p.pieces()]
    assert abs(areas[0] - (math.pi * A * A - seg)) < 1e-13
    assert abs(areas[1] - 0.5 * math.pi * (A * A - d * d)) < 1e-13
    nt, nph, nr, ns = 12, 24, 4, 24
    _, yg, _ = O.gamma_nodes(p, nt, nph)
    Am, _ = O.assemble(p, data, nr, ns, nt, nph, O.dirichlet(data, yg), rtol=1e-8)
    pan = O.panels(p, nr, ns)
    assert abs(pan["area"].sum() - sum(areas)) < 1e-12
    assert pan["area"].max() / pan["area"].min() < 20
    assert np.linalg.cond(Am) < 100


def test_piece_below_layout_resolution_gets_no_panels():
    """A ball that grazes a second face (centre 0.2999 from it: a slice of
    radius 0.0077, area about 1e-4) has two pieces, but the grazed one is
    smaller than area(S) / (nr^2 ns) and gets no sector: every panel lies on
    the top face, the panels' area is the top piece's closed-form area, and the
    collocation matrix stays well conditioned (its rings would otherwise be
    slivers of 1e-7 in area)."""
    d = 0.2999
    geo, data = _geo(), _data()
    p = O.patch_frame(geo, (2.0, 1.0 + d, 1.7), A)
    assert p.kind == 2 and p.npiece == 2
    seg = A * A * math.acos(d / A) - d * math.sqrt(A * A - d * d)
    areas = [pc[2] for pc in p.pieces()]
    assert abs(areas[0] - (math.pi * A * A - seg)) < 1e-13
    nr, ns, nt, nph = 4, 24, 12, 24
    pan = O.panels(p, nr, ns)
    assert areas[1] < sum(areas) / (nr * nr * ns)
    assert abs(pan["area"].sum() - areas[0]) < 1e-12
    assert {tuple(np.round(v, 12)) for v in pan["normal"]} == {(0.0, 0.0, -1.0)}
    _, yg, _ = O.gamma_nodes(p, nt, nph)
    Am, _ = O.assemble(p, data, nr, ns, nt, nph, O.dirichlet(data, yg), rtol=1e-8)
    assert np.linalg.cond(Am) < 100
