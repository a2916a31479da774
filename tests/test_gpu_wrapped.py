"""GPU parity on wrapped wire patches (a ball about a point of a wire face that
meets further faces of that wire, reading R15): the patch setup (hemisphere
nodes with theta_max(phi), the face pieces' panels), the assembly of Eq.
bw49-bw51 and the solve with exact values at the nodes (FP64 and mixed
precision, in a batch that mixes flat and wrapped patches), and the walks, all
against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

dtn = pytest.importorskip("paper_1210_1491_gb300")

A = 0.3
BOX = np.array([1.0, 1.0, 1.0, 3.0, 1.8, 1.7])


def _case():
    geo = W.Geometry(W.GEOM_BOX_MINUS_BOXES, lo=(0, 0, 0), hi=(4, 3, 3), boxes=np.array([BOX]))
    data = W.Dirichlet(W.DATA_POINT_SOURCE, x0=(2.0, 1.4, 1.35), strength=1.0)
    centers = np.array([[2.0, 1.4, 1.7],              # flat (top face)
                        [2.0, 1.1, 1.7],              # edge
                        [2.88, 1.65, 1.7],            # corner
                        [1.15, 1.0, 1.35],            # side face, near the end face
                        [2.4, 1.8, 1.05]])            # side face, near the bottom edge
    n = len(centers)
    batch = W.PatchBatch(centers=centers, radius=np.full(n, A), n_theta=np.full(n, 12, np.int32),
                         n_phi=np.full(n, 24, np.int32), n_rings=np.full(n, 3, np.int32),
                         n_sectors=np.full(n, 16, np.int32), walks=np.full(n, 2, np.int64))
    return W.Workload("one_wire", geo, data, batch)


def _np(t):
    return t.detach().cpu().numpy()


def _setup(wl):
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    b = wl.batch
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    return g, b, hb


def test_wrapped_setup_matches_oracle():
    wl = _case()
    g, b, hb = _setup(wl)
    r = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    assert np.all(_np(r["patch_status"]) == 0)
    P, n = 12 * 24, 3 * 16
    kinds = []
    for p in range(b.n):
        pf = O.patch_frame(wl.geometry, b.centers[p], A)
        kinds.append(pf.kind)
        _, yg, Wg = O.gamma_nodes(pf, 12, 24)
        pan = O.panels(pf, 3, 16)
        assert np.max(np.abs(_np(r["gamma_xyz"])[p * P:(p + 1) * P] - yg)) < 1e-13
        assert np.max(np.abs(_np(r["gamma_w"])[p * P:(p + 1) * P] - Wg)) < 1e-14
        assert np.max(np.abs(_np(r["colloc_xyz"])[p * n:(p + 1) * n] - pan["x"])) < 1e-13
        assert np.max(np.abs(_np(r["normals"])[p * n:(p + 1) * n] - pan["normal"])) < 1e-14
        assert np.max(np.abs(_np(r["areas"])[p * n:(p + 1) * n] - pan["area"])) < 1e-14
    assert kinds == [0, 2, 2, 2, 2]


def test_wrapped_assembly_and_solve_given_exact_values():
    """Matrix and right side against the oracle's adaptive integrals, and q:
    FP64 within relative L2 1e-10; mixed precision (a wrapped patch has a
    matrix of its own: far panels and the near panels' covers by the FP32 rule
    in offset form, the self panel by the FP64 rules; the same for its right
    side) matrix entries within 5e-7 of the largest, right side within 1e-6,
    q within 1e-5."""
    wl = _case()
    g, b, hb = _setup(wl)
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    U = O.dirichlet(wl.data, _np(r0["gamma_xyz"]))
    P, n = 12 * 24, 3 * 16
    ref = []
    for p in range(b.n):
        pf = O.patch_frame(wl.geometry, b.centers[p], A)
        Ao, bo = O.assemble(pf, wl.data, 3, 16, 12, 24, U[p * P:(p + 1) * P], rtol=1e-12)
        ref.append((Ao, bo, np.linalg.solve(Ao, bo)))
    for prec, tol in [(dtn.PREC_FP64, 1e-10), (dtn.PREC_MIXED, 1e-5)]:
        res = dtn.alloc_result(hb, want_matrix=True)
        res["u_gamma_mean"].copy_(torch.from_numpy(U))
        dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=prec, u_provided=True), result=res)
        torch.cuda.synchronize()
        assert np.all(_np(res["patch_status"]) == 0)
        for p in range(b.n):
            Ao, bo, qo = ref[p]
            Am = _np(res["matrix"])[p * n * n:(p + 1) * n * n].reshape(n, n)
            bm = _np(res["rhs"])[p * n:(p + 1) * n]
            fp64 = (prec == dtn.PREC_FP64)
            atol = 1e-10 if (fp64 or p == 0) else 5e-7          # patch 0 is flat: a shared FP64 matrix
            btol = 1e-10 if fp64 else 1e-6
            print(f"prec {prec} patch {p}: A {np.max(np.abs(Am - Ao)) / np.max(np.abs(Ao)):.1e}, "
                  f"b {np.max(np.abs(bm - bo)) / np.max(np.abs(bo)):.1e}")
            assert np.max(np.abs(Am - Ao)) <= atol * np.max(np.abs(Ao)), (prec, p)
            assert np.max(np.abs(bm - bo)) <= btol * np.max(np.abs(bo)), (prec, p)
            q = _np(res["neumann"])[p * n:(p + 1) * n]
            rel = np.linalg.norm(q - qo) / np.linalg.norm(qo)
            print(f"prec {prec} patch {p}: q rel-L2 {rel:.2e}")
            assert rel <= tol, (prec, p, rel)


def test_wrapped_walks_and_full_solve_vs_oracle():
    """Walk means at the wrapped hemisphere's nodes within 4 standard errors of
    the oracle's (FP32 walks), and the solve with the GPU's node values within
    1e-5 of the oracle's."""
    wl = _case()
    b = wl.batch
    b.walks[:] = 2000
    g, b, hb = _setup(wl)
    r = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=3))
    torch.cuda.synchronize()
    assert np.all(_np(r["patch_status"]) == 0)
    U, SE, yg = _np(r["u_gamma_mean"]), _np(r["u_gamma_se"]), _np(r["gamma_xyz"])
    q = _np(r["neumann"])
    P, n = 12 * 24, 3 * 16
    for p in (1, 2):
        sl = slice(p * P, (p + 1) * P)
        nodes = np.arange(0, P, 6)
        ro = O.wos_points(wl.geometry, wl.data, yg[sl][nodes], nodes, p, 2000,
                          O.wos_opts(eps=1e-4, seed=3, stream=O.STREAM_F32))
        Uo, SEo = O.wos_estimates(ro, 2000)
        assert np.all(np.abs(U[sl][nodes] - Uo) <= 4.0 * np.sqrt(SE[sl][nodes] ** 2 + SEo ** 2))
        rq = O.solve_patch(wl.geometry, wl.data, b.centers[p], A, 12, 24, 3, 16, 0, 0, O.wos_opts(), U_in=U[sl],
                           rtol=1e-10)
        assert np.linalg.norm(q[p * n:(p + 1) * n] - rq["q"]) / np.linalg.norm(rq["q"]) <= 1e-5


def test_wire_layout_batch_mixed_flat_and_wrapped_graph_replay():
    """The wire workload's own patches (mostly wrapped), in one mixed-precision
    call captured as a CUDA graph: the replay is bit-equal, every patch solves,
    and sampled wrapped patches match the oracle's solve with the GPU's node
    values within 1e-5."""
    wl = W.wires(n_patches=64, walks=256)
    g, b, hb = _setup(wl)
    o = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=wl.epsilon, seed=wl.seed, graph_capture=True)
    r1 = dtn.solve_patches(g, b.centers, b.radius, hb, o)
    torch.cuda.synchronize()
    q1 = _np(r1["neumann"]).copy()
    r2 = dtn.solve_patches(g, b.centers, b.radius, hb, o)
    torch.cuda.synchronize()
    assert np.array_equal(_np(r2["neumann"]), q1)
    assert np.all(_np(r2["patch_status"]) == 0)
    assert np.sum(wl.faces_met > 1) > 32
    U = _np(r2["u_gamma_mean"])
    Pn = (b.n_theta * b.n_phi).astype(np.int64)
    nn = (b.n_rings * b.n_sectors).astype(np.int64)
    goff, poff = np.r_[0, np.cumsum(Pn)], np.r_[0, np.cumsum(nn)]
    for p in [int(i) for i in np.nonzero(wl.faces_met > 1)[0][:3]]:
        rq = O.solve_patch(wl.geometry, wl.data, b.centers[p], A, int(b.n_theta[p]), int(b.n_phi[p]),
                           int(b.n_rings[p]), int(b.n_sectors[p]), 0, 0, O.wos_opts(), U_in=U[goff[p]:goff[p + 1]],
                           rtol=1e-10)
        qq = q1[poff[p]:poff[p + 1]]
        assert np.linalg.norm(qq - rq["q"]) / np.linalg.norm(rq["q"]) <= 1e-5, p


def test_mixed_batch_of_wrapped_patches_only():
    """A mixed-precision batch of wrapped patches only (no flat patch, so no
    shared right-side weights at all) solves, and gives each patch the same q,
    bit for bit, as the batch that also holds a flat patch."""
    wl = _case()
    g, b, hb = _setup(wl)
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    U = O.dirichlet(wl.data, _np(r0["gamma_xyz"]))
    o = dtn.solve_opts(prec=dtn.PREC_MIXED, u_provided=True)
    res = dtn.alloc_result(hb)
    res["u_gamma_mean"].copy_(torch.from_numpy(U))
    dtn.solve_patches(g, b.centers, b.radius, hb, o, result=res)
    P, n = 12 * 24, 3 * 16
    idx = np.arange(1, b.n)
    hb2 = dtn.HostBatch(b.n_theta[idx], b.n_phi[idx], b.n_rings[idx], b.n_sectors[idx], b.walks[idx])
    res2 = dtn.alloc_result(hb2)
    res2["u_gamma_mean"].copy_(torch.from_numpy(U[P:]))
    dtn.solve_patches(g, b.centers[idx], b.radius[idx], hb2, o, result=res2)
    torch.cuda.synchronize()
    assert np.all(_np(res2["patch_status"]) == 0)
    assert np.array_equal(_np(res2["neumann"]), _np(res["neumann"])[n:])


def test_wire_layout_wrapped_patches_match_oracle_entrywise():
    """Wrapped patches of the wire workload itself (2 to 4 faces, polar origins
    moved onto near sides among them), solved with the exact values at the GPU's
    hemisphere nodes: FP64 matrix and right side within 1e-10 of their largest
    entries and q within relative L2 1e-10 of the oracle's adaptive integrals
    and solve; mixed precision within 5e-7 (matrix), 1e-6 (right side) and
    1e-5 (q)."""
    wl = W.wires(n_patches=64, walks=64)
    idx = [int(i) for i in np.nonzero(wl.faces_met > 1)[0][:6]]
    b0 = wl.batch
    sub = W.PatchBatch(centers=b0.centers[idx], radius=b0.radius[idx], n_theta=b0.n_theta[idx],
                       n_phi=b0.n_phi[idx], n_rings=b0.n_rings[idx], n_sectors=b0.n_sectors[idx],
                       walks=b0.walks[idx])
    wl = W.Workload("wire_sub", wl.geometry, wl.data, sub)
    g, b, hb = _setup(wl)
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    U = O.dirichlet(wl.data, _np(r0["gamma_xyz"]))
    Pn = (b.n_theta * b.n_phi).astype(np.int64)
    nn = (b.n_rings * b.n_sectors).astype(np.int64)
    goff, poff, moff = np.r_[0, np.cumsum(Pn)], np.r_[0, np.cumsum(nn)], np.r_[0, np.cumsum(nn * nn)]
    ref = []
    for p in range(b.n):
        pf = O.patch_frame(wl.geometry, b.centers[p], float(b.radius[p]))
        assert pf.kind == 2
        Ao, bo = O.assemble(pf, wl.data, int(b.n_rings[p]), int(b.n_sectors[p]), int(b.n_theta[p]),
                            int(b.n_phi[p]), U[goff[p]:goff[p + 1]], rtol=1e-12)
        ref.append((Ao, bo, np.linalg.solve(Ao, bo)))
    for prec, ta, tb, tq in [(dtn.PREC_FP64, 1e-10, 1e-10, 1e-10), (dtn.PREC_MIXED, 5e-7, 1e-6, 1e-5)]:
        res = dtn.alloc_result(hb, want_matrix=True)
        res["u_gamma_mean"].copy_(torch.from_numpy(U))
        dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=prec, u_provided=True), result=res)
        torch.cuda.synchronize()
        assert np.all(_np(res["patch_status"]) == 0)
        for p in range(b.n):
            Ao, bo, qo = ref[p]
            n = int(nn[p])
            Am = _np(res["matrix"])[moff[p]:moff[p + 1]].reshape(n, n)
            bm = _np(res["rhs"])[poff[p]:poff[p + 1]]
            q = _np(res["neumann"])[poff[p]:poff[p + 1]]
            assert np.max(np.abs(Am - Ao)) <= ta * np.max(np.abs(Ao)), (prec, p)
            assert np.max(np.abs(bm - bo)) <= tb * np.max(np.abs(bo)), (prec, p)
            assert np.linalg.norm(q - qo) / np.linalg.norm(qo) <= tq, (prec, p)


@pytest.mark.parametrize("data", ["harmonic", "constant"])
def test_wrapped_patches_with_other_data(data):
    """The wrapped patches of the single-wire case with harmonic-polynomial data
    (the mixed pass differences them in FP64 at each point) and with constant
    data (no data integral): FP64 and mixed-precision solves with the exact
    values at the GPU's nodes against the oracle's adaptive integrals and solve;
    constant data give q = 0."""
    wl = _case()
    if data == "harmonic":
        wl = W.Workload("one_wire_sh", wl.geometry,
                        W.Dirichlet(W.DATA_HARMONIC_SH, lmax=4, clm=W.random_clm(4, 5), center=(2.0, 1.5, 1.5),
                                    scale=2.0), wl.batch)
    else:
        wl = W.Workload("one_wire_const", wl.geometry, W.Dirichlet(W.DATA_CONSTANT, constant=2.0), wl.batch)
    g, b, hb = _setup(wl)
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    U = O.dirichlet(wl.data, _np(r0["gamma_xyz"]))
    P, n = 12 * 24, 3 * 16
    for prec, tq in [(dtn.PREC_FP64, 1e-10), (dtn.PREC_MIXED, 1e-5)]:
        res = dtn.alloc_result(hb)
        res["u_gamma_mean"].copy_(torch.from_numpy(U))
        dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=prec, u_provided=True), result=res)
        torch.cuda.synchronize()
        assert np.all(_np(res["patch_status"]) == 0)
        for p in range(1, b.n):
            q = _np(res["neumann"])[p * n:(p + 1) * n]
            if data == "constant":
                assert np.max(np.abs(q)) < 1e-9, (prec, p)
                continue
            pf = O.patch_frame(wl.geometry, b.centers[p], A)
            Ao, bo = O.assemble(pf, wl.data, 3, 16, 12, 24, U[p * P:(p + 1) * P], rtol=1e-12)
            qo = np.linalg.solve(Ao, bo)
            assert np.linalg.norm(q - qo) / np.linalg.norm(qo) <= tq, (prec, p)
