"""dtn_wos_points_noalloc, the walk-estimate entry point for callers that cannot
allocate device memory (latency-bound serving loops, hosts that own the
device memory pool).  It must give the same estimates as
dtn_wos_points, through the C ABI, on two calls in a row (the scratch array it
reuses keeps the previous call's contents, which must not leak into the next
result), and reject sizes beyond its fixed scratch before any device work.

This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

dtn = pytest.importorskip("paper_1210_1491_gb300")


def _case():
    wl = W.unit_ball(n_patches=4)
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    y = W.targets_in_ball(700, 1.0, 0.01, seed=31)
    return g, y


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    g, y = _case()
    p = dtn.PREC_MIXED if prec == "mixed" else dtn.PREC_FP64
    opts = dtn.solve_opts(prec=p, epsilon=1e-4, seed=11)
    walks = np.full(len(y), 600, dtype=np.int64)
    walks[::7] = 1001            # uneven walk counts, ragged last chunks
    ref = dtn.wos_points(g, y, np.arange(len(y)), 5, walks, opts)
    for _ in range(2):
        out = dtn.wos_points_noalloc(g, y, np.arange(len(y)), 5, walks, opts)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out["mean"].cpu().numpy(), ref["mean"].cpu().numpy(), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(out["se"].cpu().numpy(), ref["se"].cpu().numpy(), rtol=1e-12, atol=1e-14)
        assert np.array_equal(out["steps"].cpu().numpy(), ref["steps"].cpu().numpy())
        assert np.array_equal(out["capped"].cpu().numpy(), ref["capped"].cpu().numpy())


def test_noalloc_rejects_oversized_requests():
    g, _ = _case()
    L = dtn.load()
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4)
    n = 65537
    walks = np.full(n, 16, dtype=np.int64)
    dummy = C.c_void_p(1)   # never dereferenced: the size check comes first
    rc = L.dtn_wos_points_noalloc(g.handle, n, dummy, dummy, dummy, walks.ctypes.data_as(C.c_void_p),
                                  C.byref(opts), dummy, None, None, None, None)
    assert rc == 1


def test_noalloc_call_takes_no_device_memory():
    """With the caller's tensors made beforehand, a call (after the first one on
    the device, which may load the library's module and its scratch array)
    leaves the free device memory unchanged: nothing is allocated."""
    g, y = _case()
    L = dtn.load()
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-4, seed=2)
    n = len(y)
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    pid = torch.full((n,), 9, dtype=torch.int32, device="cuda")
    walks = np.full(n, 500, dtype=np.int64)
    outs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2)]
    st = torch.empty(n, dtype=torch.int64, device="cuda")
    cp = torch.empty(n, dtype=torch.int32, device="cuda")

    def call():
        rc = L.dtn_wos_points_noalloc(g.handle, n, C.c_void_p(yd.data_ptr()), C.c_void_p(ids.data_ptr()),
                                      C.c_void_p(pid.data_ptr()), walks.ctypes.data_as(C.c_void_p), C.byref(opts),
                                      C.c_void_p(outs[0].data_ptr()), C.c_void_p(outs[1].data_ptr()),
                                      C.c_void_p(st.data_ptr()), C.c_void_p(cp.data_ptr()), None)
        assert rc == 0
        torch.cuda.synchronize()

    call()
    first = outs[0].clone()
    free0 = torch.cuda.mem_get_info()[0]
    call()
    call()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    assert torch.equal(outs[0], first)
