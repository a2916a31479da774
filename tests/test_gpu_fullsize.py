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
        assert np.all(np.abs(z) <= 4.5)
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
        assert np.all(np.abs(U[sl] - Uo) <= 4.5 * np.sqrt(SE[sl] ** 2 + SEo ** 2))
        rq = O.solve_patch(wl.geometry, wl.data, b.centers[p], 0.3, 8, 8, 4, 8, 0, 0, O.wos_opts(), U_in=U[sl],
                           rtol=1e-11)
        assert np.linalg.norm(q[p * 32:(p + 1) * 32] - rq["q"]) / np.linalg.norm(rq["q"]) <= 1e-4
