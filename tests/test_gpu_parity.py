"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Bars: Philox words and uniforms bit-exact; walk means
within 4 standard errors of the oracle's (and of the exact solution plus the
epsilon-shell bias); FP64 Neumann data within relative L2 1e-10 and mixed
precision within 1e-4 given identical hemisphere values; potential within
1e-12 (FP64) / 1e-6 (mixed); panel ownership bit-exact."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

dtn = pytest.importorskip("paper_1210_1491_gb300")


def _geom(wl):
    return dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)


def _hb(b):
    return dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks, patch_id_base=b.patch_id_base)


def _np(t):
    return t.detach().cpu().numpy()


def test_philox_bit_exact():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4099, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    seed = 0xA4093822 | (0x299F31D0 << 32)
    out = dtn.philox(ctr, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in list(range(0, 4099, 97)) + [4098]:
        assert list(out[i]) == list(O.philox(ctr[i], key))
    kat = dtn.philox(np.array([[0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]], dtype=np.uint32), seed)
    assert list(kat[0]) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_fp32_draws_bit_exact():
    """The FP32 walks' fields and uniforms equal the oracle's stream 1 bit for
    bit; their jump directions agree with the oracle's FP64 directions from the
    same uniforms to the FP32 sine/cosine accuracy."""
    rng = np.random.default_rng(3)
    n = 5003
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    seed = 0x0123456789ABCDEF
    f, u, d = dtn.philox_fields21(ctr, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    worst = 0.0
    for i in list(range(0, n, 11)) + [1, n - 1]:
        w = O.philox(ctr[i], key)
        fo = O.fields21(w)
        assert f[i].tolist() == fo.tolist()
        uo = np.array([O.u01_21(int(v)) for v in fo])
        assert np.array_equal(u[i].astype(np.float64), uo)   # exact: 22-bit odd multiples of 2^-22
        for h in range(3):
            om = O.direction(uo[2 * h], uo[2 * h + 1], O.STREAM_F32)
            worst = max(worst, float(np.max(np.abs(d[i, h].astype(np.float64) - om))))
    # FP32 z is exact; the SFU sine/cosine of an argument in (-pi, pi) and the
    # reciprocal square root are good to a few 1e-7
    assert worst < 4e-6, worst


def _wire_geometry():
    boxes = np.array([[0.3, 0.3, 0.3, 0.6, 0.5, 0.45], [0.1, 0.6, 0.6, 0.9, 0.8, 0.7],
                      [0.7, 0.1, 0.1, 0.9, 0.2, 0.9]])
    return W.Geometry(W.GEOM_BOX_MINUS_BOXES, lo=(0, 0, 0), hi=(1, 1, 1), boxes=boxes)


@pytest.mark.parametrize("kind", ["ball", "box", "wires"])
def test_distance_parity(kind):
    rng = np.random.default_rng(1)
    if kind == "ball":
        geo = W.Geometry(W.GEOM_BALL_INTERIOR, center=(0.1, 0.2, -0.1), radius=1.3)
        x = np.array(geo.center) + W.targets_in_ball(3000, 1.3, 1e-3, seed=2)
    elif kind == "box":
        geo = W.Geometry(W.GEOM_BOX_INTERIOR, lo=(0, 0, 0), hi=(1, 2, 0.5))
        x = rng.uniform((0, 0, 0), (1, 2, 0.5), (3000, 3))
    else:
        geo = _wire_geometry()
        x = rng.uniform(0, 1, (6000, 3))
        inside = np.zeros(len(x), bool)
        for b in geo.boxes:
            inside |= np.all((x > b[:3]) & (x < b[3:]), axis=1)
        x = x[~inside]
    g = dtn.Geometry.from_spec(geo, cell_size=0.05)
    d, nb = dtn.distance(g, x, prec=dtn.PREC_FP64)
    d32, nb32 = dtn.distance(g, x, prec=dtn.PREC_MIXED)
    do, nbo = O.distance(geo, x)
    d, nb, d32 = _np(d), _np(nb), _np(d32)
    if kind == "wires":
        # the grid caps distances far from all obstacles; exact below the cap
        near = do < 0.05
        assert np.all(d <= do + 1e-15)
        assert np.max(np.abs(d[near] - do[near])) < 1e-15
        assert np.max(np.abs(nb[near] - nbo[near])) < 1e-15
    else:
        assert np.max(np.abs(d - do)) < 1e-15
        assert np.max(np.abs(nb - nbo)) < 1e-14
    assert np.max(np.abs(d32 - d)) < 1e-5


def test_dirichlet_parity():
    wl = W.unit_ball(n_patches=4)
    g = _geom(wl)
    x = W.targets_in_ball(500, 1.0, 0.0, seed=7)
    v = _np(dtn.eval_dirichlet(g, x))
    vo = O.dirichlet(wl.data, x)
    assert np.max(np.abs(v - vo)) < 1e-12 * np.max(np.abs(vo))


@pytest.mark.parametrize("which", ["disk", "cap"])
def test_patch_setup_parity(which):
    if which == "disk":
        wl = W.cube_single_patch(walks=2, n_theta=9, n_phi=13, n_rings=5, n_sectors=7)
    else:
        wl = W.unit_ball(n_patches=37, walks=2, n_theta=7, n_phi=11, n_rings=6, n_sectors=5)
    g = _geom(wl)
    hb = _hb(wl.batch)
    r = dtn.solve_patches(g, wl.batch.centers, wl.batch.radius, hb,
                          dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    nt, nph, nr, ns = (int(wl.batch.n_theta[0]), int(wl.batch.n_phi[0]), int(wl.batch.n_rings[0]),
                       int(wl.batch.n_sectors[0]))
    for p in range(wl.batch.n):
        pf = O.patch_frame(wl.geometry, wl.batch.centers[p], wl.batch.radius[p])
        _, yg, Wg = O.gamma_nodes(pf, nt, nph)
        pan = O.panels(pf, nr, ns)
        P, n = nt * nph, nr * ns
        assert np.max(np.abs(_np(r["gamma_xyz"])[p * P:(p + 1) * P] - yg)) < 1e-14
        assert np.max(np.abs(_np(r["gamma_w"])[p * P:(p + 1) * P] - Wg)) < 1e-15
        assert np.max(np.abs(_np(r["colloc_xyz"])[p * n:(p + 1) * n] - pan["x"])) < 1e-14
        assert np.max(np.abs(_np(r["normals"])[p * n:(p + 1) * n] - pan["normal"])) < 1e-14
        assert np.max(np.abs(_np(r["areas"])[p * n:(p + 1) * n] - pan["area"])) < 1e-16
    assert np.all(_np(r["patch_status"]) == 0)


def _wos_case(kind):
    if kind == "cube":
        wl = W.cube_single_patch()
        y = W.points_in_box(40, (0.3, 0.3, 0.0005), (0.7, 0.7, 0.1), margin=0.0, seed=11)
    elif kind == "ball":
        wl = W.unit_ball(n_patches=4)
        y = W.targets_in_ball(40, 1.0, 0.01, seed=12)
    else:
        geo = _wire_geometry()
        data = W.Dirichlet(W.DATA_POINT_SOURCE, x0=(0.45, 0.4, 0.375))
        wl = W.Workload("wires_small", geo, data, None)
        y = W.points_in_box(400, (0.02, 0.02, 0.02), (0.98, 0.98, 0.98), margin=0.0, seed=13)
        inside = np.zeros(len(y), bool)
        for b in geo.boxes:
            inside |= np.all((y > b[:3] - 0.02) & (y < b[3:] + 0.02), axis=1)
        y = y[~inside][:40]
    return wl, y


@pytest.mark.parametrize("kind", ["cube", "ball", "wires"])
def test_wos_fp64_matches_oracle_streams(kind):
    wl, y = _wos_case(kind)
    g = dtn.Geometry.from_spec(wl.geometry, cell_size=0.05).set_data_spec(wl.data)
    N = 3000   # several chunks of 256 walks and a ragged tail
    opts = dtn.solve_opts(prec=dtn.PREC_FP64, epsilon=1e-4, seed=5)
    r = dtn.wos_points(g, y, np.arange(len(y)), 77, N, opts)
    ro = O.wos_points(wl.geometry, wl.data, y, np.arange(len(y)), 77, N,
                      O.wos_opts(eps=1e-4, seed=5, stream=O.STREAM_F64))
    Uo, SEo = O.wos_estimates(ro, N)
    U, SE = _np(r["mean"]), _np(r["se"])
    assert np.all(np.abs(U - Uo) <= 4 * np.sqrt(SE ** 2 + SEo ** 2) + 1e-12)
    if kind != "wires":
        # same Philox streams and exact distances in FP64: nearly every node follows
        # the oracle's walks.  (In the wire region the lookup grid caps the sphere
        # radius away from obstacles, a different but equally valid walk.)
        close = np.abs(U - Uo) <= 1e-9 * np.maximum(1.0, np.abs(Uo))
        assert close.mean() >= 0.9
        st = _np(r["steps"]).astype(np.int64)
        assert np.mean(np.abs(st - ro["steps"].astype(np.int64)) <= 2) >= 0.9


@pytest.mark.parametrize("kind", ["cube", "ball"])
def test_wos_fp32_follows_oracle_stream1(kind):
    """FP32 walks draw the oracle's stream-1 numbers, so with two walks per node
    nearly every node's walks are the oracle's: the same number of steps, and a
    mean that differs by the FP32 rounding of the positions and the score only.
    (Walks part where an FP32 distance falls on the other side of epsilon from
    the FP64 one, about once per 1e2 walks.)"""
    wl, _ = _wos_case(kind)
    if kind == "cube":
        y = W.points_in_box(3000, (0.05, 0.05, 0.05), (0.95, 0.95, 0.95), margin=0.0, seed=21)
        scale = 1.0 / (4 * math.pi * 0.3)
    else:
        y = W.targets_in_ball(3000, 1.0, 0.02, seed=22)
        scale = float(np.max(np.abs(O.dirichlet(wl.data, y))))
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    N = 2
    r = dtn.wos_points(g, y, np.arange(len(y)), 41, N, dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=6))
    ro = O.wos_points(wl.geometry, wl.data, y, np.arange(len(y)), 41, N,
                      O.wos_opts(eps=1e-4, seed=6, stream=O.STREAM_F32))
    Uo, _ = O.wos_estimates(ro, N)
    U = _np(r["mean"])
    same = _np(r["steps"]).astype(np.int64) == ro["steps"].astype(np.int64)
    assert same.mean() >= 0.9, same.mean()
    close = np.abs(U - Uo) <= 1e-4 * scale
    assert np.mean(close[same]) >= 0.99
    assert np.all(_np(r["capped"]) == 0)


@pytest.mark.parametrize("kind", ["cube", "ball", "wires"])
def test_wos_mixed_vs_oracle_and_exact(kind):
    wl, y = _wos_case(kind)
    g = dtn.Geometry.from_spec(wl.geometry, cell_size=0.05).set_data_spec(wl.data)
    N = 4000
    r = dtn.wos_points(g, y, np.arange(len(y)), 3, N, dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=9))
    ro = O.wos_points(wl.geometry, wl.data, y, np.arange(len(y)), 3, N,
                      O.wos_opts(eps=1e-4, seed=9, stream=O.STREAM_F32))
    Uo, SEo = O.wos_estimates(ro, N)
    U, SE = _np(r["mean"]), _np(r["se"])
    z = (U - Uo) / np.sqrt(SE ** 2 + SEo ** 2)
    assert np.all(np.abs(z) <= 4)
    ue = O.dirichlet(wl.data, y)
    L = 50.0 * np.sum(np.abs(wl.data.clm)) if kind == "ball" else 1.0 / (4 * math.pi * 0.05 ** 2)
    assert np.all(np.abs(U - ue) <= 4 * SE + 1e-4 * L)
    assert np.all(_np(r["capped"]) == 0)


def _exact_U(wl, r):
    return O.dirichlet(wl.data, _np(r["gamma_xyz"]))


@pytest.mark.parametrize("which", ["disk", "cap"])
def test_assembly_and_solve_parity_given_U(which):
    if which == "disk":
        wl = W.cube_single_patch(walks=2)
    else:
        wl = W.unit_ball(n_patches=50, walks=2, n_theta=12, n_phi=16, n_rings=8, n_sectors=8)
        wl.batch = wl.batch.subset([3, 41])
    g = _geom(wl)
    hb = _hb(wl.batch)
    # node positions first, then exact u there as the "walk" values
    r0 = dtn.solve_patches(g, wl.batch.centers, wl.batch.radius, hb,
                           dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    U = _exact_U(wl, r0)
    for prec, tol in [(dtn.PREC_FP64, 1e-10), (dtn.PREC_MIXED, 1e-4)]:
        res = dtn.alloc_result(hb, want_matrix=True)
        res["u_gamma_mean"].copy_(torch.from_numpy(U))
        dtn.solve_patches(g, wl.batch.centers, wl.batch.radius, hb,
                          dtn.solve_opts(prec=prec, u_provided=True), result=res)
        torch.cuda.synchronize()
        nt, nph, nr, ns = (int(wl.batch.n_theta[0]), int(wl.batch.n_phi[0]), int(wl.batch.n_rings[0]),
                           int(wl.batch.n_sectors[0]))
        n, P = nr * ns, nt * nph
        for p in range(wl.batch.n):
            pf = O.patch_frame(wl.geometry, wl.batch.centers[p], wl.batch.radius[p])
            Ao, bo = O.assemble(pf, wl.data, nr, ns, nt, nph, U[p * P:(p + 1) * P], rtol=1e-13)
            A = _np(res["matrix"])[p * n * n:(p + 1) * n * n].reshape(n, n)
            b = _np(res["rhs"])[p * n:(p + 1) * n]
            # the matrix uses the FP64 rules in both modes (mixed precision shares one
            # matrix per patch shape); entries agree to ~1e-12 of the largest
            assert np.max(np.abs(A - Ao)) <= 1e-11 * np.max(np.abs(Ao))
            if prec == dtn.PREC_FP64:
                assert np.max(np.abs(b - bo)) <= 1e-11 * np.max(np.abs(bo))
            else:
                assert np.max(np.abs(b - bo)) <= 1e-6 * np.max(np.abs(bo))
            qo = np.linalg.solve(Ao, bo)
            q = _np(res["neumann"])[p * n:(p + 1) * n]
            rel = np.linalg.norm(q - qo) / np.linalg.norm(qo)
            assert rel <= tol, (prec, p, rel)
        assert np.all(_np(res["patch_status"]) == 0)


def test_full_patch_with_walks_vs_oracle():
    """Steps 1 and 2 on the GPU vs the oracle with the same Philox streams (FP64)."""
    wl = W.cube_single_patch(walks=1500, n_theta=8, n_phi=8, n_rings=4, n_sectors=8)
    g = _geom(wl)
    hb = _hb(wl.batch)
    r = dtn.solve_patches(g, wl.batch.centers, wl.batch.radius, hb,
                          dtn.solve_opts(prec=dtn.PREC_FP64, epsilon=1e-4, seed=0))
    torch.cuda.synchronize()
    ro = O.solve_patch(wl.geometry, wl.data, wl.batch.centers[0], 0.1, 8, 8, 4, 8, 1500, 0,
                       O.wos_opts(eps=1e-4, seed=0), rtol=1e-12)
    U, SE = _np(r["u_gamma_mean"]), _np(r["u_gamma_se"])
    assert np.all(np.abs(U - ro["U"]) <= 4 * np.sqrt(SE ** 2 + ro["SE"] ** 2) + 1e-12)
    rq = O.solve_patch(wl.geometry, wl.data, wl.batch.centers[0], 0.1, 8, 8, 4, 8, 0, 0, O.wos_opts(),
                       U_in=U, rtol=1e-12)
    q = _np(r["neumann"])
    assert np.linalg.norm(q - rq["q"]) / np.linalg.norm(rq["q"]) < 1e-10
    assert int(_np(r["gamma_steps"]).sum()) > 64 * 1500


def test_uneven_batch_equals_alone_and_oracle():
    """Patches of different node, panel and walk counts in one launch give the
    same results as alone (bitwise: per-node fixed-point sums, per-patch ids)."""
    wl = W.unit_ball(n_patches=300, walks=600)
    sel = [5, 77, 140, 222]
    b = wl.batch.subset(sel)
    b.n_theta = np.array([6, 8, 10, 7], np.int32)
    b.n_phi = np.array([8, 12, 9, 16], np.int32)
    b.n_rings = np.array([4, 6, 3, 5], np.int32)
    b.n_sectors = np.array([8, 5, 11, 6], np.int32)
    b.walks = np.array([600, 333, 1100, 257], np.int64)
    pids = np.array(sel, np.uint32)
    g = _geom(wl)
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=1)
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks, patch_ids=pids)
    r = dtn.solve_patches(g, b.centers, b.radius, hb, opts)
    torch.cuda.synchronize()
    q_all, u_all = _np(r["neumann"]), _np(r["u_gamma_mean"])
    po = go = 0
    for k in range(4):
        hk = dtn.HostBatch(b.n_theta[k:k + 1], b.n_phi[k:k + 1], b.n_rings[k:k + 1], b.n_sectors[k:k + 1],
                           b.walks[k:k + 1], patch_ids=pids[k:k + 1])
        rk = dtn.solve_patches(g, b.centers[k:k + 1], b.radius[k:k + 1], hk, opts)
        torch.cuda.synchronize()
        n = int(b.n_rings[k] * b.n_sectors[k])
        P = int(b.n_theta[k] * b.n_phi[k])
        assert np.array_equal(_np(rk["neumann"]), q_all[po:po + n])
        assert np.array_equal(_np(rk["u_gamma_mean"]), u_all[go:go + P])
        # oracle: walks with the same streams, then the solve with the GPU's U
        ro = O.wos_points(wl.geometry, wl.data, _np(r["gamma_xyz"])[go:go + P], np.arange(P), int(pids[k]),
                          int(b.walks[k]), O.wos_opts(eps=1e-4, seed=1, stream=O.STREAM_F32))
        Uo, SEo = O.wos_estimates(ro, int(b.walks[k]))
        SE = _np(r["u_gamma_se"])[go:go + P]
        assert np.all(np.abs(u_all[go:go + P] - Uo) <= 4 * np.sqrt(SE ** 2 + SEo ** 2))
        rq = O.solve_patch(wl.geometry, wl.data, b.centers[k], 0.1, int(b.n_theta[k]), int(b.n_phi[k]),
                           int(b.n_rings[k]), int(b.n_sectors[k]), 0, 0, O.wos_opts(), U_in=u_all[go:go + P],
                           rtol=1e-12)
        assert np.linalg.norm(q_all[po:po + n] - rq["q"]) / np.linalg.norm(rq["q"]) < 1e-4
        po += n
        go += P


def test_empty_batch_and_unsupported_patch():
    wl = W.cube_single_patch(walks=64, n_theta=4, n_phi=4, n_rings=2, n_sectors=4)
    g = _geom(wl)
    empty = dtn.HostBatch(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    r = dtn.solve_patches(g, np.zeros((0, 3)), np.zeros(0), empty, dtn.solve_opts(),
                          result=dict(u_gamma_mean=torch.zeros(1, dtype=torch.float64, device="cuda"),
                                      neumann=torch.zeros(1, dtype=torch.float64, device="cuda")))
    # centre off the boundary, and a ball that reaches a second face
    c = np.array([[0.5, 0.5, 0.2], [0.05, 0.5, 0.0], [0.5, 0.5, 0.0]])
    b = dtn.HostBatch([4] * 3, [4] * 3, [2] * 3, [4] * 3, [64] * 3)
    r = dtn.solve_patches(g, c, np.full(3, 0.1), b, dtn.solve_opts(epsilon=1e-4))
    torch.cuda.synchronize()
    st = _np(r["patch_status"])
    assert st[0] == 6 and st[1] == 6 and st[2] == 0
    assert np.all(np.isfinite(_np(r["neumann"])))


def test_large_panel_count_global_lu():
    """384 panels: factors do not fit in shared memory (global-scratch LU)."""
    wl = W.cube_single_patch(walks=2, n_theta=6, n_phi=6, n_rings=16, n_sectors=24)
    g = _geom(wl)
    hb = _hb(wl.batch)
    r0 = dtn.solve_patches(g, wl.batch.centers, wl.batch.radius, hb,
                           dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    U = _exact_U(wl, r0)
    for prec in (dtn.PREC_FP64, dtn.PREC_MIXED):
        res = dtn.alloc_result(hb, want_matrix=True)
        res["u_gamma_mean"].copy_(torch.from_numpy(U))
        dtn.solve_patches(g, wl.batch.centers, wl.batch.radius, hb, dtn.solve_opts(prec=prec, u_provided=True),
                          result=res)
        torch.cuda.synchronize()
        A = _np(res["matrix"]).reshape(384, 384)
        q = _np(res["neumann"])
        b = _np(res["rhs"])
        assert np.linalg.norm(A @ q - b) <= 1e-9 * np.linalg.norm(b)


def test_potential_parity():
    rng = np.random.default_rng(3)
    npan, nt = 3001, 1000
    y = rng.uniform(-1, 1, (npan, 3))
    nrm = rng.standard_normal((npan, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    ar = rng.uniform(1e-4, 1e-3, npan)
    q = rng.standard_normal(npan)
    gv = rng.standard_normal(npan)
    t = rng.uniform(-1.5, 1.5, (nt, 3))
    ref = O.potential(y, nrm, ar, q, gv, t)
    g = dtn.Geometry(dtn.GEOM_BALL_INTERIOR, radius=1.0).set_dirichlet(dtn.DATA_CONSTANT, constant=0.0)
    u64 = _np(dtn.eval_potential(g, y, nrm, ar, q, gv, t, prec=dtn.PREC_FP64))
    u32 = _np(dtn.eval_potential(g, y, nrm, ar, q, gv, t, prec=dtn.PREC_MIXED))
    assert np.linalg.norm(u64 - ref) <= 1e-12 * np.linalg.norm(ref)
    # FP32 pair terms: positions are FP32 offsets from a tile origin (|offset| <= 4
    # here), so t - y carries an absolute error of a few eps32 * 4 and a term's
    # relative error is at most ~ eps32 (8 + 48 / r); the bound sums that over the
    # terms of each target
    d = t[:, None, :] - y[None]
    r = np.linalg.norm(d, axis=2)
    terms = np.abs(ar * q / (4 * np.pi * r)) + np.abs(ar * gv * np.einsum("tpk,pk->tp", d, nrm) / (4 * np.pi * r ** 3))
    bound = (np.finfo(np.float32).eps * terms * (8 + 48 / r)).sum(axis=1)
    assert np.all(np.abs(u32 - ref) <= bound)
    # smooth data (a harmonic potential from a patch cover) reaches 1e-6 relative
    assert np.linalg.norm(u32 - ref) <= 1e-4 * np.linalg.norm(ref)


def test_potential_parity_smooth_cover():
    """Eq. bw03 on a unit-sphere panel cover with exact data: GPU FP64 and mixed vs
    the oracle on identical panels (1e-12 / 1e-6 relative)."""
    wl = W.unit_ball(n_patches=300, a=0.25)
    xs, ns, ar = [], [], []
    for c in wl.batch.centers:
        p = O.patch_frame(wl.geometry, c, 0.25)
        pan = O.panels(p, 6, 8)
        xs.append(pan["x"]); ns.append(pan["normal"]); ar.append(pan["area"])
    xs, ns, ar = map(np.concatenate, (xs, ns, ar))
    g = O.dirichlet(wl.data, xs)
    q = O.neumann_exact(wl.data, xs, ns)
    t = W.targets_in_ball(2000, 1.0, 0.2, seed=9)
    ref = O.potential(xs, ns, ar, q, g, t)
    gg = _geom(wl)
    u64 = _np(dtn.eval_potential(gg, xs, ns, ar, q, g, t, prec=dtn.PREC_FP64))
    u32 = _np(dtn.eval_potential(gg, xs, ns, ar, q, g, t, prec=dtn.PREC_MIXED))
    assert np.linalg.norm(u64 - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.linalg.norm(u32 - ref) <= 1e-6 * np.linalg.norm(ref)


def test_gather_owned_bit_exact():
    wl = W.unit_ball(n_patches=500, a=0.2)
    g = _geom(wl)
    hb = dtn.HostBatch(wl.batch.n_theta[:500] * 0 + 2, wl.batch.n_phi * 0 + 2, wl.batch.n_rings,
                       wl.batch.n_sectors, wl.batch.walks)
    r = dtn.solve_patches(g, wl.batch.centers, np.full(500, 0.2), hb,
                          dtn.solve_opts(prec=dtn.PREC_FP64, u_provided=True))
    torch.cuda.synchronize()
    x = _np(r["colloc_xyz"])
    owner = np.repeat(np.arange(500), 128)
    keep, kept, nk = dtn.gather_owned(x, owner, wl.batch.centers)
    ko = O.owned(x, owner, wl.batch.centers)
    assert np.array_equal(_np(keep).astype(bool), ko)
    assert int(_np(nk)[0]) == int(ko.sum())
    assert np.array_equal(_np(kept)[:int(ko.sum())], np.nonzero(ko)[0])
