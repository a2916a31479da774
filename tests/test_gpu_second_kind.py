"""Second-kind local BIE on flat patches (Eq. bw55-bw59) through the C ABI
against the oracle's rows, with the exact solution on the hemisphere and with
walks."""
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
    wl = W.wires(n_patches=6, walks=400)
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


def test_caps_are_refused():
    wl = W.unit_ball(n_patches=2, walks=2)
    g, b, hb = _setup(wl)
    with pytest.raises(dtn.DtnError):
        dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_MIXED, u_provided=True, bie_kind=1))
