"""Single-point Neumann data on a flat boundary (Sec. 4.1, Eq. bw64-bw88)
through the C ABI against the oracle and the paper's Test 1: the half space
above a plane with a unit charge at depth 1, x = (0.5, 0, 0), exact q = 0.71554."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

dtn = pytest.importorskip("paper_1210_1491_gb300")

X = np.array([[0.5, 0.0, 0.0]])
Q_EXACT = 0.71554


def _np(t):
    return t.detach().cpu().numpy()


def _half_space():
    geom, data = W.half_space_charge()
    g = dtn.Geometry.from_spec(geom).set_data_spec(data)
    return geom, data, g


def test_half_space_distance_parity():
    geom, _, g = _half_space()
    pts = np.array([[0.3, -0.2, 0.7], [10.0, 3.0, 1e-3], [-4.0, 2.0, 123.0]])
    for prec in (dtn.PREC_FP64, dtn.PREC_MIXED):
        d, nb = dtn.distance(g, pts, prec=prec)
        do, nbo = O.distance(geom, pts)
        tol = 0 if prec == dtn.PREC_FP64 else 1e-6
        assert np.all(np.abs(_np(d) - do) <= tol * np.maximum(1.0, np.abs(do)))
        assert np.allclose(_np(nb), nbo, rtol=0, atol=1e-5 if tol else 0)


def test_sigma2_and_fp64_walks_match_oracle():
    geom, data, g = _half_space()
    a, ng1, ng2, walks = 0.5, 6, 20, 400
    opts = dtn.solve_opts(prec=dtn.PREC_FP64, epsilon=1e-5, seed=3)
    r = dtn.single_point_neumann(g, X, a, ng1, ng2, 1e-6 * a, walks, opts, patch_id_base=11, want_nodes=True)
    torch.cuda.synchronize()
    ro = O.single_point(geom, data, X[0], a, ng1, ng2, 1e-6 * a, walks=walks, patch=11,
                        opts=O.wos_opts(eps=1e-5, seed=3, stream=O.STREAM_F64))
    assert int(_np(r["status"])[0]) == 0
    # Sigma2' is deterministic quadrature: FP64 parity
    assert abs(_np(r["sigma2"])[0] - ro["sigma2"]) <= 1e-12 * abs(ro["sigma2"])
    # the same Philox streams from the same nodes: node means follow the oracle's
    U = _np(r["U"])
    close = np.abs(U - ro["U"]) <= 1e-9 * np.maximum(1.0, np.abs(ro["U"]))
    assert close.mean() >= 0.9
    assert abs(_np(r["sigma1"])[0] - ro["sigma1"]) <= 4 * ro["se"] + 1e-12
    assert abs(_np(r["se"])[0] - ro["se"]) <= 0.05 * ro["se"]


def test_mixed_walks_recover_test1_neumann():
    """20 x 20 hemisphere nodes (the quadrature is then exact to 6e-6), FP32
    walks: q within 4 standard errors (plus the shell and truncation bias) of
    the analytic value, and Sigma1' against the oracle's exact-solution sum."""
    geom, data, g = _half_space()
    for a in (0.1, 0.5, 1.0):
        opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-5, seed=1)
        r = dtn.single_point_neumann(g, X, a, 20, 20, 1e-6 * a, 1000, opts)
        torch.cuda.synchronize()
        q, se = _np(r["q"])[0], _np(r["se"])[0]
        assert se > 0
        assert abs(q - Q_EXACT) <= 4 * se + 2e-4, (a, q, se)
        pf = O.patch_frame(geom, X[0], a)
        _, yg, _ = O.gamma_nodes(pf, 20, 20)
        r0 = O.single_point(geom, data, X[0], a, 20, 20, 1e-6 * a, U_in=O.dirichlet(data, yg.reshape(-1, 3)))
        assert abs(_np(r["sigma1"])[0] - r0["sigma1"]) <= 4 * se + 2e-4
        # the ring rule's innermost nodes (rho ~ delta) amplify rounding of g(y) - g(x)
        assert abs(_np(r["sigma2"])[0] - r0["sigma2"]) <= 1e-12 * max(1.0, abs(r0["sigma2"]))


def test_box_face_point_and_unsupported_points():
    """A point at the centre of a face of the unit cube (point-source data, exact
    Neumann known) and, in one batch, a point whose ball reaches a second face
    (status DTN_E_UNSUPPORTED, q = 0)."""
    wl = W.cube_single_patch()
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    pts = np.array([[0.5, 0.5, 0.0], [0.05, 0.5, 0.0]])
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-5, seed=2)
    r = dtn.single_point_neumann(g, pts, 0.1, 16, 20, 1e-7, 2000, opts)
    torch.cuda.synchronize()
    st = _np(r["status"])
    assert st[0] == 0 and st[1] != 0 and _np(r["q"])[1] == 0.0
    qe = O.neumann_exact(wl.data, pts[:1], [[0, 0, -1]])[0]
    q, se = _np(r["q"])[0], _np(r["se"])[0]
    assert abs(q - qe) <= 4 * se + 1e-3 * abs(qe), (q, qe, se)


def test_invalid_arguments():
    _, _, g = _half_space()
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-5)
    with pytest.raises(dtn.DtnError):
        dtn.single_point_neumann(g, X, 0.5, 6, 6, 0.6, 100, opts)     # delta >= a
    with pytest.raises(dtn.DtnError):
        dtn.single_point_neumann(g, X, 0.5, 65, 6, 1e-6, 100, opts)   # order > 64
    with pytest.raises(dtn.DtnError):
        dtn.single_point_neumann(g, X, 0.5, 6, 6, 1e-6, 1, opts)      # < 2 walks


def test_thin_disk_distance_parity():
    geom, data = W.thin_disk()
    g = dtn.Geometry.from_spec(geom).set_data_spec(data)
    pts = np.array([[0.3, 0.4, 0.2], [3.0, 4.0, 1.0], [0.0, -2.0, -0.5], [0.99, 0.0, 1e-3]])
    do, nbo = O.distance(geom, pts)
    d, nb = dtn.distance(g, pts, prec=dtn.PREC_FP64)
    assert np.allclose(_np(d), do, rtol=1e-14, atol=1e-15) and np.allclose(_np(nb), nbo, rtol=1e-14, atol=1e-15)
    d, nb = dtn.distance(g, pts, prec=dtn.PREC_MIXED)
    assert np.allclose(_np(d), do, rtol=1e-6, atol=1e-6)


def test_thin_disk_test4_density():
    """Test 4 (Table 5): the thin disk of radius 1 at potential 1, the point
    (-0.5, 0, 0), a = 0.4, 20 x 20 nodes, 1000 walks per node (4e5 paths):
    q within 4 standard errors (plus the shell bias) of sigma(0.5) = 0.735105;
    FP64 walks follow the oracle's Philox streams."""
    geom, data = W.thin_disk()
    g = dtn.Geometry.from_spec(geom).set_data_spec(data)
    x = np.array([[-0.5, 0.0, 0.0]])
    r = dtn.single_point_neumann(g, x, 0.4, 20, 20, 4e-7, 1000,
                                 dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-5, seed=4))
    torch.cuda.synchronize()
    q, se = _np(r["q"])[0], _np(r["se"])[0]
    assert int(_np(r["status"])[0]) == 0 and abs(_np(r["sigma2"])[0]) < 1e-15
    assert abs(q - 0.735105) <= 4 * se + 2e-4, (q, se)
    r64 = dtn.single_point_neumann(g, x, 0.4, 6, 6, 4e-7, 200, dtn.solve_opts(prec=dtn.PREC_FP64, epsilon=1e-5, seed=4),
                                   patch_id_base=9, want_nodes=True)
    torch.cuda.synchronize()
    ro = O.single_point(geom, data, x[0], 0.4, 6, 6, 4e-7, walks=200, patch=9,
                        opts=O.wos_opts(eps=1e-5, seed=4, stream=O.STREAM_F64))
    close = np.abs(_np(r64["U"]) - ro["U"]) <= 1e-9 * np.maximum(1.0, np.abs(ro["U"]))
    assert close.mean() >= 0.9
