"""Fast multipole evaluation of the potential (Sec. 6: one FMM application
after the patch solves) against the oracle's direct sum of Eq. bw03.

The FMM approximates that sum; its error is bounded per target by
  trunc(t) = (1+th) th^(P+1)/(1-th) B0(t) + (1+th)^2 (P+1) th^P/(1-th)^2 B1(t)
  B0 = sum_p |c_p| / |t - y_p|,  B1 = sum_p |d_p| / |t - y_p|^2
(c_p, d_p the panel charges and dipoles) plus FP32 rounding,
  round(t) = 2 (P+1)^2 u M(t),  M = (1+th)/(1-th) B0 + ((1+th)/(1-th))^2 B1,  u = 2^-24.
Derivation: for an accepted pair (r_T + r_S < th R) the FMM keeps exactly the
terms of bidegree (j <= P, n <= P) of the expansion of 1/|t - y| in u = t - z and
v = y - c; by Banach's theorem on symmetric multilinear forms the derivatives
of 1/r satisfy |D^N(1/r)[a_1..a_N]| <= N!/r^(N+1), so the (j, n) term is at most
C(j+n, j)|u|^j |v|^n / R^(j+n+1); the dropped terms have j + n > P and sum to at
most th^(P+1)/(R(1-th)); a dipole differentiates in v (factor n); and
R >= |t - y|/(1+th).  M bounds the sum of the magnitudes of all terms, and
(P+1)^2 is the length of the longest FP32 sum (M2L).
"""
import numpy as np
import pytest
import torch

import paper_1210_1491_gb300 as dtn
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _np(x):
    torch.cuda.synchronize()
    return x.detach().cpu().numpy()


def _geom():
    return dtn.Geometry(dtn.GEOM_BALL_INTERIOR, radius=1.0).set_dirichlet(dtn.DATA_CONSTANT, constant=0.0)


def _abs_sums(y, area, q, g, t):
    return O.potential_majorants(y, area, q, g, t)


def _tolerance(b0, b1, order, theta):
    trunc = ((1 + theta) * theta ** (order + 1) / (1 - theta) * b0
             + (1 + theta) ** 2 * (order + 1) * theta ** order / (1 - theta) ** 2 * b1)
    k = (1 + theta) / (1 - theta)
    return trunc + 2 * (order + 1) ** 2 * U32 * (k * b0 + k * k * b1)


def _case(name):
    if name == "sphere":
        y, nrm, ar = W.sphere_panels(20_000)
        t = W.targets_in_ball(3000, 1.0, 0.01, seed=3)
    else:
        y, nrm, ar = W.box_surface_panels(W.wire_layout(12), 0.12)
        t = W.points_in_box(3000, (0, 0, 0), (64, 64, 16), 0.0, seed=5)
    q, g = W.panel_values(len(y))
    return y, nrm, ar, q, g, t


@pytest.mark.parametrize("name", ["sphere", "wires"])
def test_fmm_within_error_bound_and_converges(name):
    y, nrm, ar, q, g, t = _case(name)
    ref = O.potential(y, nrm, ar, q, g, t)
    b0, b1 = _abs_sums(y, ar, q, g, t)
    geom = _geom()
    for theta in (0.3, 0.5, 0.7):
        prev = None
        for order in (2, 4, 6, 8, 10, 12, 16):
            o = dtn.fmm_opts(order=order, theta=theta, leaf_sources=64, leaf_targets=64)
            u, st = dtn.eval_potential_fmm(geom, y, nrm, ar, q, g, t, opts=o, want_stats=True)
            u = _np(u)
            err = np.abs(u - ref)
            assert np.all(err <= _tolerance(b0, b1, order, theta)), (theta, order, np.max(err / _tolerance(b0, b1, order, theta)))
            rel = np.linalg.norm(u - ref) / np.linalg.norm(ref)
            # geometric decay while truncation dominates rounding
            if prev is not None and prev > 1e-5:
                assert rel <= 0.6 * prev, (theta, order, rel, prev)
            prev = rel
            assert st["m2l_pairs"] > 0 and st["p2p_pairs"] > 0
            assert st["source_levels"] >= 3 and st["target_levels"] >= 3


def test_fmm_single_leaf_is_the_direct_sum():
    # every cell a leaf: the traversal gives one leaf pair, evaluated by FP32 pair
    # terms from FP32 offsets to the leaf centre (|offset| <= 2 here); the bound is
    # the one of the direct FP32 sum
    y, nrm, ar = W.sphere_panels(3000)
    q, g = W.panel_values(3000)
    t = W.targets_in_ball(2000, 1.0, 0.02, seed=8)
    ref = O.potential(y, nrm, ar, q, g, t)
    o = dtn.fmm_opts(order=4, theta=0.5, leaf_sources=4096, leaf_targets=4096)
    u, st = dtn.eval_potential_fmm(_geom(), y, nrm, ar, q, g, t, opts=o, want_stats=True)
    u = _np(u)
    assert st["m2l_pairs"] == 0 and st["p2p_pairs"] == 1 and st["p2p_terms"] == 3000 * 2000
    d = t[:, None, :] - y[None]
    r = np.linalg.norm(d, axis=2)
    terms = np.abs(ar * q / (4 * np.pi * r)) + np.abs(ar * g * np.einsum("tpk,pk->tp", d, nrm) / (4 * np.pi * r ** 3))
    bound = (np.finfo(np.float32).eps * terms * (8 + 48 / r)).sum(axis=1)
    assert np.all(np.abs(u - ref) <= bound)


def test_fmm_panel_index_and_data_paths():
    y, nrm, ar = W.sphere_panels(12_000)
    q, g = W.panel_values(12_000)
    t = W.targets_in_ball(1500, 1.0, 0.02, seed=10)
    geom = _geom()
    o = dtn.fmm_opts(order=8, theta=0.5, leaf_sources=32, leaf_targets=48)
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(12_000, 7000, replace=False))
    full = _np(dtn.eval_potential_fmm(geom, y[idx], nrm[idx], ar[idx], q[idx], g[idx], t, opts=o))
    cnt = torch.tensor([7000], dtype=torch.int64, device="cuda")
    via = _np(dtn.eval_potential_fmm(geom, y, nrm, ar, q, g, t, opts=o, index=idx, n_index=cnt))
    # entries past the count are never read
    idx_long = np.concatenate([idx, np.full(12_000 - 7000, 10 ** 9, dtype=np.int64)])
    via_long = _np(dtn.eval_potential_fmm(geom, y, nrm, ar, q, g, t, opts=o, index=idx_long, n_index=cnt))
    assert np.array_equal(full, via) and np.array_equal(full, via_long)
    # without a count the index holds one entry per panel row (a permutation here)
    perm = rng.permutation(12_000)
    a = _np(dtn.eval_potential_fmm(geom, y[perm], nrm[perm], ar[perm], q[perm], g[perm], t, opts=o))
    b = _np(dtn.eval_potential_fmm(geom, y, nrm, ar, q, g, t, opts=o, index=perm))
    assert np.array_equal(a, b)
    with pytest.raises(ValueError):
        dtn.eval_potential_fmm(geom, y, nrm, ar, q, g, t, opts=o, index=idx)
    # an index outside the panel arrays is found on the device, before any read
    bad = idx.copy()
    bad[17] = 12_000
    with pytest.raises(dtn.DtnError):
        dtn.eval_potential_fmm(geom, y, nrm, ar, q, g, t, opts=o, index=bad, n_index=cnt)
    bad[17] = -1
    with pytest.raises(dtn.DtnError):
        dtn.eval_potential_fmm(geom, y, nrm, ar, q, g, t, opts=o, index=bad, n_index=cnt)
    # dirichlet=None: g from the data set on the geometry (a point source)
    x0 = np.array([0.3, -0.2, 1.7])
    gp = dtn.Geometry(dtn.GEOM_BALL_INTERIOR, radius=1.0).set_dirichlet(dtn.DATA_POINT_SOURCE, x0=x0, strength=1.0)
    gv = _np(dtn.eval_dirichlet(gp, y))
    a = _np(dtn.eval_potential_fmm(gp, y, nrm, ar, q, None, t, opts=o))
    b = _np(dtn.eval_potential_fmm(gp, y, nrm, ar, q, gv, t, opts=o))
    assert np.array_equal(a, b)


def test_fmm_reproduces_harmonic_field_inside_ball():
    # exact Dirichlet and Neumann data of a point source outside the unit ball:
    # the representation returns u inside (discretisation error of the
    # equal-area midpoint rule, O(h^2)), and the FMM stays within its bound of
    # the direct sum
    y, nrm, ar = W.sphere_panels(200_000)
    x0 = np.array([0.4, 0.3, 1.6])
    r = y - x0
    dist = np.linalg.norm(r, axis=1)
    gval = 1.0 / (4 * np.pi * dist)
    qval = -np.einsum("pk,pk->p", r, nrm) / (4 * np.pi * dist ** 3)
    t = W.targets_in_ball(400, 1.0, 0.3, seed=12)
    o = dtn.fmm_opts(order=10, theta=0.5)
    u = _np(dtn.eval_potential_fmm(_geom(), y, nrm, ar, qval, gval, t, opts=o))
    exact = 1.0 / (4 * np.pi * np.linalg.norm(t - x0, axis=1))
    assert np.linalg.norm(u - exact) <= 1e-3 * np.linalg.norm(exact)
    ref = O.potential(y, nrm, ar, qval, gval, t)
    b0, b1 = _abs_sums(y, ar, qval, gval, t)
    assert np.all(np.abs(u - ref) <= _tolerance(b0, b1, 10, 0.5))


def test_fmm_edge_cases():
    geom = _geom()
    o = dtn.fmm_opts(order=6, theta=0.5, leaf_sources=16, leaf_targets=16)
    t = W.targets_in_ball(300, 1.0, 0.0, seed=2)
    # no panels: zero potential
    z = _np(dtn.eval_potential_fmm(geom, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0),
                                   np.zeros(0), t, opts=o))
    assert np.array_equal(z, np.zeros(300))
    # no targets
    y, nrm, ar = W.sphere_panels(500)
    q, g = W.panel_values(500)
    e = _np(dtn.eval_potential_fmm(geom, y, nrm, ar, q, g, np.zeros((0, 3)), opts=o))
    assert e.shape == (0,)
    # one panel, targets far away (a single accepted pair high in the trees)
    far = W.targets_in_ball(200, 1.0, 0.0, seed=6) + np.array([40.0, 0.0, 0.0])
    for srcs in (1, 500):
        ref = O.potential(y[:srcs], nrm[:srcs], ar[:srcs], q[:srcs], g[:srcs], far)
        u = _np(dtn.eval_potential_fmm(geom, y[:srcs], nrm[:srcs], ar[:srcs], q[:srcs], g[:srcs], far, opts=o))
        b0, b1 = _abs_sums(y[:srcs], ar[:srcs], q[:srcs], g[:srcs], far)
        assert np.all(np.abs(u - ref) <= _tolerance(b0, b1, 6, 0.5))
    # repeated panel points: cells stop at max_level with more than leaf_sources points
    rep = np.repeat(y[:40], 50, axis=0)
    rn = np.repeat(nrm[:40], 50, axis=0)
    ra = np.repeat(ar[:40], 50)
    rq, rg = W.panel_values(2000, seed=4)
    o2 = dtn.fmm_opts(order=8, theta=0.5, leaf_sources=8, leaf_targets=8, max_level=6)
    ref = O.potential(rep, rn, ra, rq, rg, t)
    u, st = dtn.eval_potential_fmm(geom, rep, rn, ra, rq, rg, t, opts=o2, want_stats=True)
    u = _np(u)
    b0, b1 = _abs_sums(rep, ra, rq, rg, t)
    assert st["source_levels"] == 7
    assert np.all(np.abs(u - ref) <= _tolerance(b0, b1, 8, 0.5))
    # invalid options
    for bad in (dict(order=0), dict(order=17), dict(theta=0.0), dict(theta=1.0), dict(leaf_sources=0),
                dict(leaf_targets=5000), dict(max_level=0), dict(max_level=22)):
        kw = dict(order=6, theta=0.5, leaf_sources=16, leaf_targets=16, max_level=20)
        kw.update(bad)
        with pytest.raises(dtn.DtnError):
            dtn.eval_potential_fmm(geom, y, nrm, ar, q, g, t, opts=dtn.fmm_opts(**kw))


def test_fmm_full_size_sampled():
    # 1e6 panels on the unit sphere and 1e6 targets in the ball, the size the
    # direct sum stops being practical at; 1500 sampled targets against the oracle
    n = 1_000_000
    y, nrm, ar = W.sphere_panels(n)
    q, g = W.panel_values(n)
    t = W.targets_in_ball(n, 1.0, 0.0, seed=4)
    geom = _geom()
    o = dtn.fmm_opts(order=10, theta=0.5)
    dev = [torch.tensor(a, device="cuda") for a in (y, nrm, ar, q, g, t)]
    u, st = dtn.eval_potential_fmm(geom, *dev, opts=o, want_stats=True)
    u = _np(u)
    again, st2 = dtn.eval_potential_fmm(geom, *dev, opts=o, want_stats=True)
    assert np.array_equal(u, _np(again))   # deterministic: sorted lists, fixed sum order
    # list capacities grown by a first call are kept by the geometry's workspace
    assert st["source_levels"] >= 7 and st2["restarts"] == 0
    assert {k: v for k, v in st.items() if k != "restarts"} == {k: v for k, v in st2.items() if k != "restarts"}
    sample = np.random.default_rng(1).choice(n, 1500, replace=False)
    ref = O.potential(y, nrm, ar, q, g, t[sample])
    b0, b1 = _abs_sums(y, ar, q, g, t[sample])
    assert np.all(np.abs(u[sample] - ref) <= _tolerance(b0, b1, 10, 0.5))


@pytest.mark.parametrize("order,theta,ls,lt,ml", [
    (1, 0.3, 16, 16, 20),      # lowest order: the bound is loose, the traversal the same
    (16, 0.7, 64, 64, 20),     # highest order
    (6, 0.05, 8, 8, 20),       # theta near 0: almost every pair is a leaf pair
    (12, 0.95, 32, 32, 20),    # theta near 1: the slowest convergence the acceptance allows
    (8, 0.5, 1, 1, 20),        # one point per leaf (deep trees)
    (8, 0.5, 4096, 4096, 20),  # one leaf each: a single leaf pair
    (8, 0.5, 8, 8, 1),         # max_level 1: leaves of any size at level 1
])
def test_fmm_option_extremes(order, theta, ls, lt, ml):
    # two clusters of panels (one dense) and targets around and between them
    y1, n1, a1 = W.sphere_panels(3000, radius=0.2)
    y2, n2, a2 = W.sphere_panels(800, radius=1.0)
    y = np.concatenate([y1 + np.array([0.6, 0.0, 0.0]), y2])
    nrm = np.concatenate([n1, n2])
    ar = np.concatenate([a1, a2])
    q, g = W.panel_values(len(y), seed=21)
    t = np.concatenate([W.targets_in_ball(700, 1.0, 0.05, seed=22),
                        W.targets_outside_ball(300, 1.0, 0.1, seed=23)])
    ref = O.potential(y, nrm, ar, q, g, t)
    b0, b1 = _abs_sums(y, ar, q, g, t)
    o = dtn.fmm_opts(order=order, theta=theta, leaf_sources=ls, leaf_targets=lt, max_level=ml)
    u, st = dtn.eval_potential_fmm(_geom(), y, nrm, ar, q, g, t, opts=o, want_stats=True)
    u = _np(u)
    assert np.all(np.isfinite(u))
    assert np.all(np.abs(u - ref) <= _tolerance(b0, b1, order, theta))
    assert st["source_levels"] <= ml + 1 and st["target_levels"] <= ml + 1
    if ls == 4096:
        assert st["m2l_pairs"] == 0 and st["p2p_pairs"] == 1


def test_fmm_wires_full_size_sampled():
    # 2.1e6 square panels on the faces of the 200-wire layout (h = 0.05) and 1e6
    # targets in the outer box: deep, uneven source trees (9 levels); 600
    # sampled targets against the oracle within the bound
    boxes = W.wire_layout(200)
    y, nrm, ar = W.box_surface_panels(boxes, 0.05)
    q, g = W.panel_values(len(y), seed=5)
    t = W.points_in_box(1_000_000, (0, 0, 0), (64, 64, 16), 0.0, seed=6)
    dev = [torch.tensor(a, device="cuda") for a in (y, nrm, ar, q, g, t)]
    o = dtn.fmm_opts(order=10, theta=0.6, leaf_sources=128, leaf_targets=64)
    u, st = dtn.eval_potential_fmm(_geom(), *dev, opts=o, want_stats=True)
    u = _np(u)
    assert st["source_levels"] >= 8 and st["m2l_pairs"] > 10 ** 6
    sample = np.random.default_rng(2).choice(len(t), 600, replace=False)
    ref = O.potential(y, nrm, ar, q, g, t[sample])
    b0, b1 = _abs_sums(y, ar, q, g, t[sample])
    assert np.all(np.abs(u[sample] - ref) <= _tolerance(b0, b1, 10, 0.6))
