"""Continuous-batching server: queries submitted while others run are admitted
as slots and device memory free up, overlap on the device (CUDA events on the
slot streams), and give the same result alone, in a mix and through a direct
dtn_solve_patches call (bitwise: every random number is fixed by the patch id
and the walk sums are per-node fixed point).  A failing patch is reported with
its query and does not disturb the others; a query that cannot fit the memory
budget is refused with DTN_E_OUT_OF_MEMORY."""
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
        assert r is not None and r["status"] == 0, r
        assert np.all(r["patch_status"] == 0)
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


def _heavy_queries(n_q=6):
    """Queries big enough (about 10 ms of walks each) that batches of two slots
    meet on the device."""
    wl = W.unit_ball(n_patches=400, walks=2048)
    qs = []
    for k in range(n_q):
        idx = np.arange(20 * k, 20 * k + 20)
        qs.append(dict(centers=wl.batch.centers[idx], radius=wl.batch.radius[idx],
                       n_theta=np.full(20, 16), n_phi=np.full(20, 16), n_rings=np.full(20, 4),
                       n_sectors=np.full(20, 8), walks=np.full(20, 2048), patch_ids=idx.astype(np.uint32)))
    return wl, qs


def test_batches_overlap_on_the_device_and_results_do_not_change():
    """Two slots sharing the SMs: the device intervals (events around each batch
    on its slot stream) intersect, and every query's result is bit-equal to its
    result served alone."""
    wl, qs = _heavy_queries()
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=4)
    srv = dtn.Server(g, opts, max_inflight=2, max_batch_patches=20, split_sms=True)
    alone = [_run(srv, [q])[0] for q in qs]
    st0 = srv.stats()
    mix = _run(srv, qs)
    st = srv.stats()
    srv.close()
    for a, m in zip(alone, mix):
        assert np.array_equal(a["neumann"], m["neumann"])
        assert np.array_equal(a["u"], m["u"])
    assert st["batches"] == st0["batches"] + len(qs)
    assert st["max_concurrent"] >= 2
    assert st["overlap_ms"] > st0["overlap_ms"]
    assert 0 < st["budget_bytes"] <= st["device_free_bytes"]
    assert st["peak_held_bytes"] <= st["budget_bytes"]
    print(f"served {len(qs)} queries: device busy {st['busy_ms'] - st0['busy_ms']:.1f} ms, "
          f"two batches in flight {st['overlap_ms'] - st0['overlap_ms']:.1f} ms")


def test_failing_patch_reported_with_its_query_only():
    """A patch whose centre is not on the boundary (unsupported, injected on the
    host) fails alone: its query reports DTN_E_UNSUPPORTED with the patch's
    status, the query's other patches and the other queries in the same batch
    keep their results."""
    wl, qs = _queries()
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=4)
    srv = dtn.Server(g, opts, max_inflight=1, max_batch_patches=64)
    alone = [_run(srv, [q])[0] for q in qs[:3]]
    bad = {k: np.array(v, copy=True) for k, v in qs[1].items()}
    bad["centers"][0] *= 0.5          # inside the ball, not on its boundary
    tickets = [srv.submit(**qs[0]), srv.submit(**bad), srv.submit(**qs[2])]
    srv.drain()
    r0, rb, r2 = (srv.poll(t) for t in tickets)
    srv.close()
    assert r0["status"] == 0 and r2["status"] == 0
    assert np.array_equal(r0["neumann"], alone[0]["neumann"])
    assert np.array_equal(r2["neumann"], alone[2]["neumann"])
    assert rb["status"] == 6                      # DTN_E_UNSUPPORTED
    assert rb["patch_status"][0] == 6 and np.all(rb["patch_status"][1:] == 0)
    n0 = int(qs[1]["n_rings"][0] * qs[1]["n_sectors"][0])
    assert np.array_equal(rb["neumann"][n0:], alone[1]["neumann"][n0:])


def test_admission_by_memory_budget():
    """A budget below one query's workspace refuses it (DTN_E_OUT_OF_MEMORY,
    counted as rejected) and leaves the server usable; a budget of a few
    queries serves them all without the ledger passing the budget."""
    wl, qs = _heavy_queries(4)
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=4)
    tiny = dtn.Server(g, opts, max_inflight=2, max_batch_patches=64, memory_budget=1 << 16)
    t = tiny.submit(**qs[0])
    tiny.drain()
    r = tiny.poll(t)
    st = tiny.stats()
    tiny.close()
    assert r["status"] == 2 and r["neumann"] is None     # DTN_E_OUT_OF_MEMORY
    assert st["rejected"] == 1 and st["budget_bytes"] == 1 << 16
    srv = dtn.Server(g, opts, max_inflight=3, max_batch_patches=64, memory_budget=200 << 20)
    out = _run(srv, qs)
    st = srv.stats()
    srv.close()
    assert len(out) == 4 and st["rejected"] == 0
    assert st["peak_held_bytes"] <= st["budget_bytes"] == 200 << 20
