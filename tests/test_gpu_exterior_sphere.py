"""The patch method outside the sphere of radius 3 (Sec. 5.2) through the C
ABI: cap patches with the signed radius, walks that escape through the
truncation sphere, the matrix, right side and solve against the oracle, and
the Neumann data against u = R/|x| (q = 1/R along the region's outward normal)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

dtn = pytest.importorskip("paper_1210_1491_gb300")
R, A = 3.0, 1.0


def _np(t):
    return t.detach().cpu().numpy()


def _case(n=8, walks=2, **kw):
    wl = W.sphere_exterior(n_patches=n, walks=walks, **kw)
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    b = wl.batch
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    return wl, g, hb


def test_distance_and_walks_vs_exact():
    wl, g, _ = _case()
    pts = np.array([[0.0, 0.0, 5.0], [4.0, 0.0, 3.0], [0.1, -3.2, 0.2]])
    d, _ = dtn.distance(g, pts, prec=dtn.PREC_FP64)
    do, _ = O.distance(wl.geometry, pts)
    assert np.allclose(_np(d), do, rtol=1e-14, atol=1e-15)
    y = np.array([[0.0, 0.0, 3.4], [2.2, 2.2, 0.5], [0.0, -4.5, 1.0]])
    exact = R / np.linalg.norm(y, axis=1)
    for prec in (dtn.PREC_MIXED, dtn.PREC_FP64):
        r = dtn.wos_points(g, y, np.arange(3), 1, 4000, dtn.solve_opts(prec=prec, epsilon=1e-4, seed=3))
        # escaped walks score 0 and count in the mean; none is cut at max_steps
        assert np.all(_np(r["capped"]) == 0)
        assert np.all(np.abs(_np(r["mean"]) - exact) <= 4 * _np(r["se"]) + 1e-3)


def test_assembly_and_solve_parity_given_exact_values():
    wl, g, hb = _case(n=8, n_theta=16, n_phi=32, n_rings=4, n_sectors=8)
    b = wl.batch
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    U = R / np.linalg.norm(_np(r0["gamma_xyz"]), axis=1)
    n, P = 32, 512
    for prec, qtol in ((dtn.PREC_FP64, 1e-10), (dtn.PREC_MIXED, 1e-4)):
        res = dtn.alloc_result(hb, want_matrix=True)
        res["u_gamma_mean"].copy_(torch.from_numpy(U))
        dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=prec, u_provided=True), result=res)
        torch.cuda.synchronize()
        assert np.all(_np(res["patch_status"]) == 0)
        for p in (0, 5):
            pf = O.patch_frame(wl.geometry, b.centers[p], A)
            Ao, bo = O.assemble(pf, wl.data, 4, 8, 16, 32, U[p * P:(p + 1) * P], rtol=1e-13)
            Am = _np(res["matrix"])[p * n * n:(p + 1) * n * n].reshape(n, n)
            bm = _np(res["rhs"])[p * n:(p + 1) * n]
            assert np.max(np.abs(Am - Ao)) <= 1e-11 * np.max(np.abs(Ao))
            btol = 1e-11 if prec == dtn.PREC_FP64 else 1e-6
            assert np.max(np.abs(bm - bo)) <= btol * np.max(np.abs(bo))
            qo = np.linalg.solve(Ao, bo)
            q = _np(res["neumann"])[p * n:(p + 1) * n]
            assert np.linalg.norm(q - qo) / np.linalg.norm(qo) <= qtol
            # the Neumann data themselves: 1/R inside r < 0.7a (Sec. 5.2 accuracy)
            prm = O.panels(pf, 4, 8)["prm"]
            inner = 2 * R * np.sin(prm[:, 4] / 2) < 0.7 * A
            assert np.max(np.abs(q[inner] * R - 1.0)) < 0.03


def test_full_solve_with_walks():
    """Walks (mixed precision) then assembly and solve; the oracle solves with
    the GPU's hemisphere estimates, and the Neumann data stay within the Monte
    Carlo error of 1/R."""
    wl, g, hb = _case(n=4, walks=2000, n_theta=16, n_phi=32, n_rings=4, n_sectors=8)
    b = wl.batch
    r = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=1))
    torch.cuda.synchronize()
    U = _np(r["u_gamma_mean"])
    ye = R / np.linalg.norm(_np(r["gamma_xyz"]), axis=1)
    # scores are 1 (absorbed on the sphere) or 0 (gone to infinity): near the
    # sphere few walks escape and the sample error can be 0, so take the larger
    # of it and the exact binomial error
    se = np.maximum(_np(r["u_gamma_se"]), np.sqrt(ye * (1 - ye) / 2000))
    assert np.all(np.abs(U - ye) <= 4 * se + 1e-3)
    n, P = 32, 512
    for p in range(2):
        ro = O.solve_patch(wl.geometry, wl.data, b.centers[p], A, 16, 32, 4, 8, 0, 0, O.wos_opts(),
                           U_in=U[p * P:(p + 1) * P], rtol=1e-12)
        q = _np(r["neumann"])[p * n:(p + 1) * n]
        assert np.linalg.norm(q - ro["q"]) / np.linalg.norm(ro["q"]) < 1e-4
