"""Oracle pins for the single-point method on a flat boundary (Sec. 4.1,
Eq. bw64-bw88): the deterministic Sigma2' quadrature against the values printed
in Tables 1 and 2, Sigma1' with the exact solution on the hemisphere against the
analytic Neumann value of Test 1, and the walks of the half-space region against
the exact solution."""
import math
import os

import numpy as np

import oracle.oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
X = np.array([0.5, 0.0, 0.0])
Q_EXACT = 0.71554   # Table 1, analytic solution (printed to 5 digits)


def _golden():
    t1, t2, sec = [], [], None
    with open(os.path.join(GOLDEN, "paper_single_point_sigma.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            if line.startswith("["):
                sec = line.split("]")[0][1:]
                continue
            v = [float(t) for t in line.split()]
            (t1 if sec == "table1" else t2).append(v)
    return t1, t2


def _exact_nodes(geom, data, a, ng1):
    pf = O.patch_frame(geom, X, a)
    _, yg, _ = O.gamma_nodes(pf, ng1, ng1)
    return O.dirichlet(data, yg.reshape(-1, 3))


def test_half_space_distance_and_frame():
    g, _ = W.half_space_charge()
    d, nb = O.distance(g, [[0.3, -0.2, 0.7]])
    assert abs(d[0] - 0.7) < 1e-15 and np.allclose(nb[0], [0.3, -0.2, 0.0])
    pf = O.patch_frame(g, X, 0.5)
    assert np.allclose(np.asarray(pf.n), [0, 0, -1])   # outward of the region z > 0
    # the hemisphere lies in the region
    _, yg, _ = O.gamma_nodes(pf, 6, 6)
    assert np.all(yg.reshape(-1, 3)[:, 2] > 0)


def test_sigma2_matches_table1():
    g, d = W.half_space_charge()
    t1, _ = _golden()
    for a, s2 in t1:
        r = O.single_point(g, d, X, a, 4, 20, 1e-6 * a, U_in=np.zeros(16))
        assert abs(r["sigma2"] - s2) <= 1e-6, (a, r["sigma2"], s2)


def test_sigma2_table2_delta_and_order():
    """Table 2's rows are reproduced by the ring rule with the Jacobian a/2 of
    the interval [delta, a] (the printed values are the (a - delta)/2 rule times
    a / (a - delta)); at delta/a <= 1e-4 the two agree to the printed digits.
    The O(delta) trend of Eq. bw82 holds for the rule as written."""
    g, d = W.half_space_charge()
    _, t2 = _golden()
    a = 0.5
    for row in t2:
        da = row[0]
        delta = da * a
        for n, printed in zip((4, 6, 10, 20), row[1:]):
            s2 = O.single_point(g, d, X, a, 4, n, delta, U_in=np.zeros(16))["sigma2"]
            assert abs(s2 * a / (a - delta) - printed) <= 6e-6, (da, n, s2, printed)
    ref = O.single_point(g, d, X, a, 4, 20, 1e-6 * a, U_in=np.zeros(16))["sigma2"]
    errs = [abs(O.single_point(g, d, X, a, 4, 20, da * a, U_in=np.zeros(16))["sigma2"] - ref)
            for da in (1e-1, 1e-2, 1e-3)]
    # error ~ C delta: each tenfold smaller delta cuts it about tenfold
    assert errs[1] < 0.2 * errs[0] and errs[2] < 0.2 * errs[1]


def test_exact_hemisphere_values_recover_analytic_neumann():
    g, d = W.half_space_charge()
    t1, _ = _golden()
    for a, _ in t1:
        U = _exact_nodes(g, d, a, 20)
        r = O.single_point(g, d, X, a, 20, 20, 1e-6 * a, U_in=U)
        assert abs(r["q"] - Q_EXACT) <= 6e-6, (a, r["q"])
        assert r["se"] == 0.0
    # the analytic value itself
    qn = O.neumann_exact(d, [X], [[0, 0, -1]])[0]
    assert abs(qn - Q_EXACT) < 5e-6


def test_sigma1_sign_and_kernel_weight():
    """Sigma1' of a constant solution vanishes, and for u linear in z (u = z + g0,
    exact q = -1 along n = -z) the hemisphere rule alone gives q (Sigma2' = 0 as
    the data are constant on the plane)."""
    g, _ = W.half_space_charge()
    const = W.Dirichlet(W.DATA_CONSTANT, constant=2.5)
    r = O.single_point(g, const, X, 0.3, 10, 10, 1e-6, U_in=np.full(100, 2.5))
    assert abs(r["q"]) < 1e-14
    pf = O.patch_frame(g, X, 0.3)
    _, yg, _ = O.gamma_nodes(pf, 10, 10)
    U = 2.5 + yg.reshape(-1, 3)[:, 2]
    r = O.single_point(g, const, X, 0.3, 10, 10, 1e-6, U_in=U)
    assert abs(r["sigma1"] - (-1.0)) < 1e-12 and abs(r["sigma2"]) < 1e-15


def test_walks_in_half_space_within_4se_of_exact():
    g, d = W.half_space_charge()
    a, ng1, walks = 0.5, 6, 600
    r = O.single_point(g, d, X, a, ng1, 20, 1e-6 * a, walks=walks, patch=3, opts=O.wos_opts(eps=1e-5))
    U = _exact_nodes(g, d, a, ng1)
    r0 = O.single_point(g, d, X, a, ng1, 20, 1e-6 * a, U_in=U)
    assert r["se"] > 0
    # shell bias O(eps |grad u|) per node, negligible at eps = 1e-5
    assert abs(r["sigma1"] - r0["sigma1"]) <= 4 * r["se"] + 1e-4, (r["sigma1"], r0["sigma1"], r["se"])
    # per-node means against the exact solution
    res = O.wos_points(g, d, O.gamma_nodes(O.patch_frame(g, X, a), ng1, ng1)[1].reshape(-1, 3)[:6],
                       np.arange(6, dtype=np.uint32), np.full(6, 3, np.uint32), np.full(6, walks, np.int64),
                       O.wos_opts(eps=1e-5))
    mean, se = O.wos_estimates(res, walks)
    assert np.all(np.abs(mean - U[:6]) <= 4 * se + 1e-4)
