"""Harmonic-polynomial Dirichlet data (real solid harmonics, Eq. bw01 with
g = sum c_lm r^l Y_lm) evaluated inside every kernel family that reads the data:
the second-kind rows on a flat patch and the single-point ring rule (Sec. 4.1),
against the oracle on the unit cube.  Each CUDA translation unit holds its own
copy of the harmonic recurrence tables, so each family is checked on its own."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

dtn = pytest.importorskip("paper_1210_1491_gb300")


def _np(t):
    return t.detach().cpu().numpy()


def _cube_with_harmonic_data():
    wl = W.cube_single_patch(walks=2, n_theta=16, n_phi=32, n_rings=8, n_sectors=8)
    data = W.Dirichlet(W.DATA_HARMONIC_SH, lmax=4, clm=W.random_clm(4, 3), center=(0.5, 0.5, 0.5), scale=1.0)
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(data)
    return wl, data, g


def test_second_kind_rows_with_harmonic_data():
    wl, data, g = _cube_with_harmonic_data()
    b = wl.batch
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    U = O.dirichlet(data, _np(r0["gamma_xyz"]).reshape(-1, 3))
    res = dtn.alloc_result(hb)
    res["u_gamma_mean"].copy_(torch.from_numpy(U))
    dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True, bie_kind=1),
                      result=res)
    torch.cuda.synchronize()
    pf = O.patch_frame(wl.geometry, b.centers[0], 0.1)
    qo = O.second_kind_flat(pf, data, 16, 32, 8, 8, U, ng2=20)
    # the two sides evaluate the harmonic data by different recurrences (equal to
    # ~1e-16 |g|); the tangential gradient takes differences over h = 1e-5 a, so
    # it differs by ~1e-16 |g| / h ~ 1e-10 |g|, and the rows by a few times that
    assert np.max(np.abs(_np(res["neumann"]) - qo)) <= 1e-9 * np.max(np.abs(qo))


def test_single_point_ring_rule_with_harmonic_data():
    wl, data, g = _cube_with_harmonic_data()
    x = np.array([[0.5, 0.5, 0.0]])
    a, ng1, ng2 = 0.1, 6, 20
    opts = dtn.solve_opts(prec=dtn.PREC_FP64, epsilon=1e-5, seed=3)
    r = dtn.single_point_neumann(g, x, a, ng1, ng2, 1e-6 * a, 20, opts)
    torch.cuda.synchronize()
    ro = O.single_point(wl.geometry, data, x[0], a, ng1, ng2, 1e-6 * a, walks=20,
                        opts=O.wos_opts(eps=1e-5, seed=3, stream=O.STREAM_F64))
    assert int(_np(r["status"])[0]) == 0
    assert abs(_np(r["sigma2"])[0] - ro["sigma2"]) <= 1e-12 * max(1.0, abs(ro["sigma2"]))


@pytest.mark.parametrize("lmax", [3, 8, 12])
def test_fp32_walk_scoring_of_harmonic_data(lmax):
    """Walks that start inside the epsilon shell of the unit ball end on their first
    step and score the data at the radial projection of the start point: the FP32
    scoring (solid-harmonic recurrence over the FP32 pair table) against the
    oracle's FP64 harmonic, for the degree-4, degree-8 and general-degree forms."""
    geom = W.Geometry(W.GEOM_BALL_INTERIOR, center=(0.0, 0.0, 0.0), radius=1.0)
    data = W.Dirichlet(W.DATA_HARMONIC_SH, lmax=lmax, clm=W.random_clm(lmax, 5), center=(0.1, -0.2, 0.05),
                       scale=1.3)
    g = dtn.Geometry.from_spec(geom).set_data_spec(data)
    rng = np.random.default_rng(11)
    u = rng.normal(size=(300, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    y = (1.0 - 5e-5) * u
    for prec in (dtn.PREC_MIXED, dtn.PREC_FP64):
        r = dtn.wos_points(g, y, np.arange(300), 0, 4, dtn.solve_opts(prec=prec, epsilon=1e-4, seed=1))
        assert np.all(_np(r["steps"]) == 4) and np.all(_np(r["capped"]) == 0)
        ref = O.dirichlet(data, u)
        err = np.max(np.abs(_np(r["mean"]) - ref)) / np.max(np.abs(ref))
        assert err <= (3e-5 if prec == dtn.PREC_MIXED else 1e-12), (prec, err)
