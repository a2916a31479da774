"""Second-kind local BIE (Eq. bw55-bw59) through the C ABI against the oracle:
flat patches (q = 2b row by row) and cap patches ((1/2 I - D) q = b), with the
exact solution on the hemisphere and with walks."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

dtn = pytest.importorskip("paper_1210_1491_gb300")


def _np(t):
    return t.detach().cpu().numpy()


def _setup(wl):
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    b = wl.batch
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    return g, b, hb


def test_rows_match_oracle_with_exact_values():
    wl = W.cube_single_patch(walks=2, n_theta=16, n_phi=32, n_rings=8, n_sectors=8)
    g, b, hb = _setup(wl)
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    U = O.dirichlet(wl.data, _np(r0["gamma_xyz"]))
    for prec in (dtn.PREC_FP64, dtn.PREC_MIXED):
        res = dtn.alloc_result(hb)
        res["u_gamma_mean"].copy_(torch.from_numpy(U))
        dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=prec, u_provided=True, bie_kind=1),
                          result=res)
        torch.cuda.synchronize()
        pf = O.patch_frame(wl.geometry, b.centers[0], 0.1)
        qo = O.second_kind_flat(pf, wl.data, 16, 32, 8, 8, U, ng2=20)
        q = _np(res["neumann"])
        assert np.max(np.abs(q - qo)) <= 1e-10 * np.max(np.abs(qo))
        assert np.all(_np(res["patch_status"]) == 0) and np.all(_np(res["refine_iters"]) == 0)
        pan = O.panels(pf, 8, 8)
        qe = O.neumann_exact(wl.data, pan["x"], pan["normal"])
        inner = np.linalg.norm(pan["Xloc"][:, :2], axis=1) < 0.07
        assert np.max(np.abs(q[inner] - qe[inner]) / np.abs(qe[inner])) < 1e-3


def test_with_walks_on_wire_patches():
    wl = W.wires(n_patches=6, walks=400, allow_wrapped=False)
    g, b, hb = _setup(wl)
    res = dtn.solve_patches(g, b.centers, b.radius, hb,
                            dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=2, bie_kind=1, ring_order=16))
    torch.cuda.synchronize()
    U = _np(res["u_gamma_mean"])
    q = _np(res["neumann"])
    go, po = 0, 0
    for p in range(2):
        nt, nph, nr, ns = (int(v[p]) for v in (b.n_theta, b.n_phi, b.n_rings, b.n_sectors))
        pf = O.patch_frame(wl.geometry, b.centers[p], float(b.radius[p]))
        qo = O.second_kind_flat(pf, wl.data, nt, nph, nr, ns, U[go:go + nt * nph], ng2=16)
        qq = q[po:po + nr * ns]
        assert np.max(np.abs(qq - qo)) <= 1e-10 * max(1.0, np.max(np.abs(qo)))
        go += nt * nph
        po += nr * ns


def _cap_case(wl, a, exact_u):
    g, b, hb = _setup(wl)
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    U = exact_u(_np(r0["gamma_xyz"]).reshape(-1, 3))
    return g, b, hb, U


@pytest.mark.parametrize("case", ["ball", "exterior"])
def test_cap_system_matches_oracle_with_exact_values(case):
    """Cap patches: (1/2 I - D) q = b, D per shape group in mixed precision.
    GPU (fixed Gauss covers of order >= 16, Duffy triangles on the self panel)
    against the oracle (adaptive rules at rtol 1e-10, a 20-point Duffy rule on
    the self panel, converged to a few 1e-12): FP64 q within relative L2 1e-10
    of the oracle's.  Mixed precision
    takes the right side by a geodesic polar rule of order 32 about x_i (order
    20: 2e-6, 32: 4e-8, 48: 4e-10 of max|b| on a unit-ball cap) applied to the
    data interpolated on each panel from its 8 x 8 samples (degree 7 per
    direction; on these coarse 4 x 8 panels a few 1e-7 of max|q|): 1e-6 of
    max|q|.  Closed forms:
    harmonic data on the unit ball (inner rows 1e-3 of max|q|), unit potential
    on the R = 3 sphere seen from outside (q = 1/R, 5e-3 inside r < 0.7a)."""
    if case == "ball":
        wl = W.unit_ball(n_patches=3, walks=2, n_theta=16, n_phi=32, n_rings=4, n_sectors=8)
        a, exact_u = 0.1, (lambda y: O.dirichlet(wl.data, y))
        inner_tol = 1e-3
    else:
        wl = W.sphere_exterior(n_patches=3, walks=2, n_theta=16, n_phi=32, n_rings=4, n_sectors=8)
        a, exact_u = 1.0, (lambda y: 3.0 / np.linalg.norm(y, axis=1))
        inner_tol = 5e-3
    g, b, hb, U = _cap_case(wl, a, exact_u)
    for prec in (dtn.PREC_FP64, dtn.PREC_MIXED):
        res = dtn.alloc_result(hb)
        res["u_gamma_mean"].copy_(torch.from_numpy(U))
        dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=prec, u_provided=True, bie_kind=1),
                          result=res)
        torch.cuda.synchronize()
        q = _np(res["neumann"])
        assert np.all(_np(res["patch_status"]) == 0)
        for p in range(3):
            pf = O.patch_frame(wl.geometry, b.centers[p], a)
            qo = O.second_kind(pf, wl.data, 16, 32, 4, 8, U[p * 512:(p + 1) * 512])
            qq = q[p * 32:(p + 1) * 32]
            if prec == dtn.PREC_FP64:
                rel = np.linalg.norm(qq - qo) / np.linalg.norm(qo)
                print(f"{case} patch {p}: FP64 rel-L2 {rel:.2e}, max-abs "
                      f"{np.max(np.abs(qq - qo)) / np.max(np.abs(qo)):.2e}")
                assert rel <= 1e-10, (p, rel)
            else:
                assert np.max(np.abs(qq - qo)) <= 1e-6 * np.max(np.abs(qo)), (prec, p)
            pan = O.panels(pf, 4, 8)
            qe = (O.neumann_exact(wl.data, pan["x"], pan["normal"]) if case == "ball" else np.full(32, 1.0 / 3.0))
            inner = np.linalg.norm(pan["Xloc"][:, :2], axis=1) < 0.7 * a
            assert np.max(np.abs(qq - qe)[inner]) <= inner_tol * np.max(np.abs(qe)), (prec, p)


def test_cap_second_kind_with_walks_against_the_oracle_and_the_first_kind():
    """200 unit-ball caps of the bench shape with 4096 walks per node: the GPU's
    second-kind solve (mixed precision: polar rule on the interpolated data,
    1e-6 as above)
    against the oracle's on the GPU's own node values (sampled patches), and the
    Neumann error against the closed form
    over whole patches no larger than the first kind's (the better-conditioned
    system keeps the rim rows)."""
    wl = W.unit_ball(n_patches=200, walks=4096)
    g, b, hb = _setup(wl)
    r2 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_MIXED, bie_kind=1, seed=1))
    r1 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_MIXED, bie_kind=0, seed=1))
    torch.cuda.synchronize()
    assert np.all(_np(r2["patch_status"]) == 0)
    U = _np(r2["u_gamma_mean"]).reshape(200, -1)
    q2 = _np(r2["neumann"]).reshape(200, -1)
    q1 = _np(r1["neumann"]).reshape(200, -1)
    xs = _np(r2["colloc_xyz"]).reshape(200, -1, 3)
    ns_ = _np(r2["normals"]).reshape(200, -1, 3)
    e1, e2 = [], []
    for p in (0, 57, 199):
        pf = O.patch_frame(wl.geometry, b.centers[p], 0.1)
        qo = O.second_kind(pf, wl.data, 16, 32, 8, 16, U[p])
        assert np.max(np.abs(q2[p] - qo)) <= 1e-6 * np.max(np.abs(qo)), p
        qe = O.neumann_exact(wl.data, xs[p], ns_[p])
        e1.append(np.linalg.norm(q1[p] - qe) / np.linalg.norm(qe))
        e2.append(np.linalg.norm(q2[p] - qe) / np.linalg.norm(qe))
    assert np.mean(e2) <= np.mean(e1)
