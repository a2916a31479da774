"""Runtime pieces around the kernels: CUDA-graph replay, the walk-kernel
autotuner, stage timing, and capped walks.  The walk estimates must not depend
on launch parameters (chunk size, resident blocks, refill threshold) nor on
graph replay: they are bitwise reproducible."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

dtn = pytest.importorskip("paper_1210_1491_gb300")


def _case():
    wl = W.unit_ball(n_patches=200, walks=700, n_theta=8, n_phi=12, n_rings=6, n_sectors=8)
    b = wl.batch.subset(np.arange(0, 200, 7))
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks, patch_ids=np.arange(0, 200, 7))
    return wl, b, g, hb


def test_results_independent_of_launch_parameters():
    wl, b, g, hb = _case()
    ref = None
    for chunk, bps, refill in [(256, 0, 8), (64, 1, 2), (512, 5, 16), (100, 7, 5)]:
        o = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=3, walk_chunk=chunk, wos_blocks_per_sm=bps,
                           wos_refill=refill)
        r = dtn.solve_patches(g, b.centers, b.radius, hb, o)
        torch.cuda.synchronize()
        out = (r["u_gamma_mean"].cpu().numpy(), r["neumann"].cpu().numpy(), r["gamma_steps"].cpu().numpy())
        if ref is None:
            ref = out
        else:
            for a, c in zip(ref, out):
                assert np.array_equal(a, c)


def test_graph_replay_matches_direct_and_stage_times():
    wl, b, g, hb = _case()
    o = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=3)
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, o)
    torch.cuda.synchronize()
    og = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=3, graph_capture=True, record_stages=True)
    res = dtn.alloc_result(hb)
    c = torch.from_numpy(b.centers).cuda()
    rad = torch.from_numpy(b.radius).cuda()
    for _ in range(3):   # capture, then two replays
        res["neumann"].zero_()
        dtn.solve_patches(g, c, rad, hb, og, result=res)
        torch.cuda.synchronize()
        assert np.array_equal(res["neumann"].cpu().numpy(), r0["neumann"].cpu().numpy())
        ms = g.stage_times()   # a replay is timed as a whole in ms[0]
        assert all(m >= 0 for m in ms) and ms[0] > 0


def test_graph_replay_second_kind_caps():
    """The second-kind path on caps (group weights, samples, product, group LU)
    captured and replayed: bit-equal to the direct call."""
    wl, b, g, hb = _case()
    o = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=3, bie_kind=1)
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, o)
    torch.cuda.synchronize()
    og = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=3, bie_kind=1, graph_capture=True)
    res = dtn.alloc_result(hb)
    c = torch.from_numpy(b.centers).cuda()
    rad = torch.from_numpy(b.radius).cuda()
    for _ in range(3):   # capture, then two replays
        res["neumann"].zero_()
        dtn.solve_patches(g, c, rad, hb, og, result=res)
        torch.cuda.synchronize()
        assert np.array_equal(res["neumann"].cpu().numpy(), r0["neumann"].cpu().numpy())
    assert np.all(res["patch_status"].cpu().numpy() == 0)


def test_autotuner_picks_and_results_unchanged():
    wl, b, g, hb = _case()
    o = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=3)
    r0 = dtn.solve_patches(g, b.centers, b.radius, hb, o)
    torch.cuda.synchronize()
    t = dtn.autotune_walks(g, b.centers, b.radius, hb, o)
    assert t["walk_chunk"] in (64, 128, 256, 512) and 5 <= t["wos_blocks_per_sm"] <= 9
    assert t["wos_refill"] in (4, 8, 12, 16) and t["ns_per_walk_step"] > 0
    r1 = dtn.solve_patches(g, b.centers, b.radius, hb, o)   # now with tuned parameters
    torch.cuda.synchronize()
    assert np.array_equal(r0["neumann"].cpu().numpy(), r1["neumann"].cpu().numpy())


def test_capped_walks_counted_and_excluded():
    wl = W.cube_single_patch(walks=200, n_theta=4, n_phi=4, n_rings=2, n_sectors=4)
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    y = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.00005]])
    for prec in (dtn.PREC_MIXED, dtn.PREC_FP64):
        r = dtn.wos_points(g, y, [0, 1], 0, 200, dtn.solve_opts(prec=prec, epsilon=1e-4, max_steps=3))
        cap = r["capped"].cpu().numpy()
        st = r["steps"].cpu().numpy()
        assert cap[0] > 0 and cap[1] == 0         # a centre walk rarely ends in 3 steps; the shell point at once
        assert st[1] == 200
        # a cut walk made exactly 3 steps, every other one 1 to 3
        assert 3 * cap[0] + (200 - cap[0]) <= st[0] <= 600


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_walk_cap_status_and_nodes_without_estimates(prec):
    """max_steps = 2: nearly every walk is cut.  Each patch reports
    DTN_E_WALK_CAP; a node keeping no walk has mean NaN and standard error
    +inf, a node keeping one walk a finite mean and +inf, and the counts add
    up (kept + cut = walks)."""
    wl = W.unit_ball(n_patches=3, walks=6, n_theta=8, n_phi=8, n_rings=4, n_sectors=8)
    b = wl.batch
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    p = dtn.PREC_MIXED if prec == "mixed" else dtn.PREC_FP64
    r = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=p, epsilon=1e-4, max_steps=2))
    torch.cuda.synchronize()
    assert np.all(r["patch_status"].cpu().numpy() == 7)   # DTN_E_WALK_CAP
    cut = r["gamma_capped"].cpu().numpy().astype(np.int64)
    kept = 6 - cut
    U = r["u_gamma_mean"].cpu().numpy()
    SE = r["u_gamma_se"].cpu().numpy()
    assert np.all((cut >= 0) & (cut <= 6)) and cut.sum() > 0
    assert np.all(np.isnan(U[kept == 0])) and np.all(np.isposinf(SE[kept == 0]))
    assert np.all(np.isfinite(U[kept == 1])) and np.all(np.isposinf(SE[kept == 1]))
    assert np.all(np.isfinite(U[kept >= 2])) and np.all(np.isfinite(SE[kept >= 2]))
    # without a cap the same batch solves cleanly
    r2 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=p, epsilon=1e-4))
    torch.cuda.synchronize()
    assert np.all(r2["patch_status"].cpu().numpy() == 0)
    assert np.all(r2["gamma_capped"].cpu().numpy() == 0)


def test_not_converged_status():
    """Mixed precision (FP32 factors, FP64-residual refinement), one sweep
    against an unreachable tolerance: every patch reports DTN_E_NOT_CONVERGED
    with its residual and sweep count, and solves cleanly with the defaults.
    The FP64 path factors in FP64 and does not refine: its status stays
    DTN_OK with 0 sweeps whatever the tolerance."""
    wl = W.unit_ball(n_patches=3, walks=2, n_theta=8, n_phi=8, n_rings=4, n_sectors=8)
    b = wl.batch
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    for p in (dtn.PREC_MIXED, dtn.PREC_FP64):
        res = dtn.alloc_result(hb)
        r0 = dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=p, u_provided=True), result=res)
        torch.cuda.synchronize()
        res["u_gamma_mean"].copy_(torch.from_numpy(O_exact(wl, r0)))
        dtn.solve_patches(g, b.centers, b.radius, hb,
                          dtn.solve_opts(prec=p, u_provided=True, max_refine_iters=1, refine_tol=1e-300), result=res)
        torch.cuda.synchronize()
        st = res["patch_status"].cpu().numpy()
        it = res["refine_iters"].cpu().numpy()
        if p == dtn.PREC_MIXED:
            assert np.all(st == 4), st   # DTN_E_NOT_CONVERGED
            assert np.all(res["residual"].cpu().numpy() > 0)
            assert np.all(it == 1)
        else:
            assert np.all(st == 0) and np.all(it == 0)
        dtn.solve_patches(g, b.centers, b.radius, hb, dtn.solve_opts(prec=p, u_provided=True), result=res)
        torch.cuda.synchronize()
        assert np.all(res["patch_status"].cpu().numpy() == 0), p


def O_exact(wl, r):
    import oracle as O
    return O.dirichlet(wl.data, r["gamma_xyz"].cpu().numpy())
