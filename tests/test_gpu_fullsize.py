"""Parity at the benchmark's full size and launch configuration: the 2000-patch
unit-ball workload (512 nodes x 4096 walks, 128 panels per patch) solved in one
mixed-precision call, then sampled patches recomputed by the oracle: walk
means within 4 standard errors of the oracle's walks on the same Philox streams,
and Neumann data within 1e-4 of the oracle's solve with the GPU's node values.
Also the wire layout (box minus 200 obstacle boxes) on a few patches."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

dtn = pytest.importorskip("paper_1210_1491_gb300")


def test_unit_ball_full_size_sampled():
    wl = W.unit_ball()   # the benchmark workload
    b = wl.batch
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    r = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=wl.epsilon,
                                                                     seed=wl.seed))
    torch.cuda.synchronize()
    st = r["patch_status"].cpu().numpy()
    assert np.all(st == 0)
    U = r["u_gamma_mean"].cpu().numpy()
    SE = r["u_gamma_se"].cpu().numpy()
    q = r["neumann"].cpu().numpy()
    yg = r["gamma_xyz"].cpu().numpy()
    P, n = 512, 128
    for p in (0, 1234):
        sl = slice(p * P, (p + 1) * P)
        # walks: a sample of 64 nodes of the patch, full walk count, same streams
        nodes = np.arange(0, P, 8)
        ro = O.wos_points(wl.geometry, wl.data, yg[sl][nodes], nodes, p, 4096,
                          O.wos_opts(eps=wl.epsilon, seed=wl.seed, stream=O.STREAM_F32))
        Uo, SEo = O.wos_estimates(ro, 4096)
        z = (U[sl][nodes] - Uo) / np.sqrt(SE[sl][nodes] ** 2 + SEo ** 2)
        print(f"patch {p}: max |z| = {np.max(np.abs(z)):.2f}")
        assert np.all(np.abs(z) <= 4.0)
        # solve: the oracle's assembly and LU with the GPU's node values
        rq = O.solve_patch(wl.geometry, wl.data, b.centers[p], 0.1, 16, 32, 8, 16, 0, 0, O.wos_opts(),
                           U_in=U[sl], rtol=1e-11)
        rel = np.linalg.norm(q[p * n:(p + 1) * n] - rq["q"]) / np.linalg.norm(rq["q"])
        assert rel <= 1e-4, rel
    # accuracy against the exact Neumann data inside r < 0.7a (discretisation + walks)
    x = r["colloc_xyz"].cpu().numpy()[: 50 * n]
    nrm = r["normals"].cpu().numpy()[: 50 * n]
    qe = O.neumann_exact(wl.data, x, nrm)
    loc = np.linalg.norm(x - np.repeat(b.centers[:50], n, axis=0), axis=1)
    inner = loc < 0.07
    err = np.linalg.norm((q[: 50 * n] - qe)[inner]) / np.linalg.norm(qe[inner])
    assert err < 0.1, err


def test_wire_patches_vs_oracle():
    wl = W.wires(n_patches=4, walks=1024)
    b = wl.batch
    b.n_theta[:] = 8
    b.n_phi[:] = 8
    b.n_rings[:] = 4
    b.n_sectors[:] = 8
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    r = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=2))
    torch.cuda.synchronize()
    assert np.all(r["patch_status"].cpu().numpy() == 0)
    U = r["u_gamma_mean"].cpu().numpy()
    SE = r["u_gamma_se"].cpu().numpy()
    yg = r["gamma_xyz"].cpu().numpy()
    q = r["neumann"].cpu().numpy()
    for p in range(2):
        sl = slice(p * 64, (p + 1) * 64)
        ro = O.wos_points(wl.geometry, wl.data, yg[sl], np.arange(64), p, 1024,
                          O.wos_opts(eps=1e-4, seed=2, stream=O.STREAM_F32))
        Uo, SEo = O.wos_estimates(ro, 1024)
        assert np.all(np.abs(U[sl] - Uo) <= 4.0 * np.sqrt(SE[sl] ** 2 + SEo ** 2))
        rq = O.solve_patch(wl.geometry, wl.data, b.centers[p], 0.3, 8, 8, 4, 8, 0, 0, O.wos_opts(), U_in=U[sl],
                           rtol=1e-11)
        assert np.linalg.norm(q[p * 32:(p + 1) * 32] - rq["q"]) / np.linalg.norm(rq["q"]) <= 1e-4


def test_precision_study_scaled_unit_ball():
    """The precision study on the scaled unit ball (2e4 patches, 256 panels,
    1024 nodes x 8192 walks): FP32 walks with FP64 sums and the FP32 shared
    factors with FP64-residual refinement over all patches in one call; the
    all-FP64 path (FP64 walks, FP64 assembly and LU, one patch per call) on a
    sample; both against the exact Neumann data and against the oracle's solve
    with their own node values.  Prints the per-patch relative L2 errors."""
    wl = W.unit_ball_scaled()
    b = wl.batch
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    r = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=wl.epsilon,
                                                                     seed=wl.seed))
    torch.cuda.synchronize()
    assert np.all(r["patch_status"].cpu().numpy() == 0)
    P, n = 1024, 256
    q = r["neumann"].cpu().numpy()
    x = r["colloc_xyz"].cpu().numpy()
    nrm = r["normals"].cpu().numpy()
    U = r["u_gamma_mean"].cpu().numpy()
    iters = r["refine_iters"].cpu().numpy()
    assert iters.max() <= 10
    sample = (0, 7777, 19999)
    errs_mixed, errs_fp64 = [], []
    for p in sample:
        sl = slice(p * n, (p + 1) * n)
        inner = np.linalg.norm(x[sl] - b.centers[p], axis=1) < 0.07
        qe = O.neumann_exact(wl.data, x[sl], nrm[sl])
        errs_mixed.append(np.linalg.norm((q[sl] - qe)[inner]) / np.linalg.norm(qe[inner]))
        # the oracle's collocation solve with the GPU's node values
        rq = O.solve_patch(wl.geometry, wl.data, b.centers[p], 0.1, 32, 32, 16, 16, 0, 0, O.wos_opts(),
                           U_in=U[p * P:(p + 1) * P], rtol=1e-10)
        assert np.linalg.norm(q[sl] - rq["q"]) / np.linalg.norm(rq["q"]) <= 1e-4
        # the all-FP64 path on the same patch (its own FP64 walks)
        h1 = dtn.HostBatch(b.n_theta[p:p + 1], b.n_phi[p:p + 1], b.n_rings[p:p + 1], b.n_sectors[p:p + 1],
                           b.walks[p:p + 1], patch_id_base=p)
        r64 = dtn.solve_patches(g, b.centers[p:p + 1], b.radius[p:p + 1], h1,
                                dtn.solve_opts(prec=dtn.PREC_FP64, epsilon=wl.epsilon, seed=wl.seed))
        torch.cuda.synchronize()
        q64 = r64["neumann"].cpu().numpy()
        errs_fp64.append(np.linalg.norm((q64 - qe)[inner]) / np.linalg.norm(qe[inner]))
    print("precision study rel-L2 (r < 0.7a) mixed:", errs_mixed, "fp64:", errs_fp64)
    # both paths sit at the Monte Carlo + discretisation level, and neither is
    # systematically worse than the other by more than that level
    assert max(errs_mixed) < 0.05 and max(errs_fp64) < 0.05
    assert np.mean(errs_mixed) < 2.0 * np.mean(errs_fp64) + 0.01


def test_wires_full_size_uneven_batch_graph_replay():
    """The batching workload at full size: 1e4 wire-face patches of uneven sizes
    (16^2..32^2 nodes, 32..512 panels, 2048 walks) in one mixed-precision call,
    captured as a CUDA graph and replayed; the replay gives the same results bit
    for bit, and sampled patches of each size match the oracle (walk means
    within 4 standard errors on the same Philox streams; the collocation solve
    within 1e-4 with the GPU's node values)."""
    wl = W.wires()
    b = wl.batch
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    o = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=wl.epsilon, seed=wl.seed, graph_capture=True)
    r1 = dtn.solve_patches(g, b.centers, b.radius, hb, o)
    torch.cuda.synchronize()
    q1 = r1["neumann"].cpu().numpy().copy()
    r2 = dtn.solve_patches(g, b.centers, b.radius, hb, o)   # replay of the captured graph
    torch.cuda.synchronize()
    assert np.array_equal(r2["neumann"].cpu().numpy(), q1)
    assert np.all(r2["patch_status"].cpu().numpy() == 0)
    U = r2["u_gamma_mean"].cpu().numpy()
    SE = r2["u_gamma_se"].cpu().numpy()
    yg = r2["gamma_xyz"].cpu().numpy()
    P = (b.n_theta * b.n_phi).astype(np.int64)
    n = (b.n_rings * b.n_sectors).astype(np.int64)
    goff = np.r_[0, np.cumsum(P)]
    poff = np.r_[0, np.cumsum(n)]
    # one sampled patch of each node order (the one with the fewest panels, to
    # keep the oracle's quadrature short)
    picks = []
    for k in np.unique(P):
        idx = np.nonzero(P == k)[0]
        picks.append(int(idx[np.argmin(n[idx])]))
    for p in picks:
        gs = slice(goff[p], goff[p + 1])
        nodes = np.arange(0, P[p], max(1, P[p] // 32))
        ro = O.wos_points(wl.geometry, wl.data, yg[gs][nodes], nodes, p, int(b.walks[p]),
                          O.wos_opts(eps=wl.epsilon, seed=wl.seed, stream=O.STREAM_F32))
        Uo, SEo = O.wos_estimates(ro, int(b.walks[p]))
        assert np.all(np.abs(U[gs][nodes] - Uo) <= 4.0 * np.sqrt(SE[gs][nodes] ** 2 + SEo ** 2))
        rq = O.solve_patch(wl.geometry, wl.data, b.centers[p], float(b.radius[p]), int(b.n_theta[p]),
                           int(b.n_phi[p]), int(b.n_rings[p]), int(b.n_sectors[p]), 0, 0, O.wos_opts(),
                           U_in=U[gs], rtol=1e-10)
        qq = q1[poff[p]:poff[p + 1]]
        assert np.linalg.norm(qq - rq["q"]) / np.linalg.norm(rq["q"]) <= 1e-4
