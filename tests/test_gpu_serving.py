"""Continuous-batching server: queries submitted while others run are admitted
as slots free up, overlap on the device, and give the same result alone, in a
mix and through a direct dtn_solve_patches call (bitwise: every random number
is fixed by the patch id and the walk sums are per-node fixed point)."""
import time

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

dtn = pytest.importorskip("paper_1210_1491_gb300")


def _queries():
    wl = W.unit_ball(n_patches=400, walks=256)
    rng = np.random.Generator(np.random.PCG64(21))
    qs = []
    start = 0
    for k in range(6):
        n = int(rng.integers(1, 12))
        idx = np.arange(start, start + n)
        start += n
        qs.append(dict(
            centers=wl.batch.centers[idx], radius=wl.batch.radius[idx],
            n_theta=np.full(n, int(rng.choice([6, 8]))), n_phi=np.full(n, 8),
            n_rings=np.full(n, int(rng.choice([3, 4]))), n_sectors=np.full(n, 8),
            walks=np.full(n, int(rng.choice([128, 300, 1000]))), patch_ids=idx.astype(np.uint32)))
    return wl, qs


def _run(srv, qs):
    tickets = [srv.submit(**q) for q in qs]
    srv.drain()
    out = []
    for t in tickets:
        r = srv.poll(t)
        assert r is not None
        out.append(r)
    return out


def test_alone_equals_mix_equals_direct():
    wl, qs = _queries()
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=4)
    srv = dtn.Server(g, opts, max_inflight=3, max_batch_patches=16)
    alone = [_run(srv, [q])[0] for q in qs]
    mix = _run(srv, qs)
    for a, m in zip(alone, mix):
        assert np.array_equal(a["neumann"], m["neumann"])
        assert np.array_equal(a["u"], m["u"])
        assert m["latency_s"] > 0
    # staggered arrivals: later queries arrive while earlier batches run
    tickets = []
    for q in qs:
        tickets.append(srv.submit(**q))
        time.sleep(0.002)
    srv.drain()
    for t, a in zip(tickets, alone):
        assert np.array_equal(srv.poll(t)["neumann"], a["neumann"])
    # direct call on the same patches
    for q, a in zip(qs, alone):
        hb = dtn.HostBatch(q["n_theta"], q["n_phi"], q["n_rings"], q["n_sectors"], q["walks"],
                           patch_ids=q["patch_ids"])
        r = dtn.solve_patches(g, q["centers"], q["radius"], hb, opts)
        torch.cuda.synchronize()
        assert np.array_equal(r["neumann"].cpu().numpy(), a["neumann"])
    srv.close()


def test_served_result_matches_oracle():
    wl, qs = _queries()
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=4)
    srv = dtn.Server(g, opts, max_inflight=2, max_batch_patches=8)
    q = qs[0]
    r = _run(srv, [q])[0]
    srv.close()
    nt, nph, nr, ns = int(q["n_theta"][0]), int(q["n_phi"][0]), int(q["n_rings"][0]), int(q["n_sectors"][0])
    P, n = nt * nph, nr * ns
    ro = O.solve_patch(wl.geometry, wl.data, q["centers"][0], 0.1, nt, nph, nr, ns, 0, 0, O.wos_opts(),
                       U_in=r["u"][:P], rtol=1e-12)
    assert np.linalg.norm(r["neumann"][:n] - ro["q"]) / np.linalg.norm(ro["q"]) < 1e-4
