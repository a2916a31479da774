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
    t1, t2, t4, sec = [], [], [], None
    with open(os.path.join(GOLDEN, "paper_single_point_sigma.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            if line.startswith("["):
                sec = line.split("]")[0][1:]
                continue
            v = [float(t) for t in line.split()]
            {"table1": t1, "table2": t2, "test4": t4}[sec].append(v)
    return t1, t2, t4


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
    t1, _, _ = _golden()
    for a, s2 in t1:
        r = O.single_point(g, d, X, a, 4, 20, 1e-6 * a, U_in=np.zeros(16))
        assert abs(r["sigma2"] - s2) <= 1e-6, (a, r["sigma2"], s2)


def test_sigma2_table2_delta_and_order():
    """Table 2's rows are reproduced by the ring rule with the Jacobian a/2 of
    the interval [delta, a] (the printed values are the (a - delta)/2 rule times
    a / (a - delta)); at delta/a <= 1e-4 the two agree to the printed digits.
    The O(delta) trend of Eq. bw82 holds for the rule as written."""
    g, d = W.half_space_charge()
    _, t2, _ = _golden()
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
    t1, _, _ = _golden()
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


def _disk_potential(p, b=1.0):
    """Potential of the thin disk of radius b at potential 1 (oblate spheroidal
    solution): u = (2/pi) asin(2b / (r1 + r2)), r1,2 = distances to the rim
    circle's nearest and farthest points in the meridian plane."""
    p = np.atleast_2d(p)
    r = np.hypot(p[:, 0], p[:, 1])
    r1 = np.hypot(r - b, p[:, 2])
    r2 = np.hypot(r + b, p[:, 2])
    return (2.0 / math.pi) * np.arcsin(np.minimum(1.0, 2.0 * b / (r1 + r2)))


def test_thin_disk_closed_form_is_the_solution():
    """The closed form used below: 1 on the disk, harmonic off it (finite
    differences), decays like 2b/(pi |x|), and its normal derivative on the disk
    is the analytic density of Test 4."""
    on = np.array([[0.3, 0.2, 0.0], [-0.9, 0.0, 0.0]])
    assert np.allclose(_disk_potential(on), 1.0, atol=1e-12)
    h = 1e-3
    for x in ([0.4, 0.3, 0.5], [1.5, -0.2, 0.1], [0.0, 0.0, 2.0]):
        x = np.array(x)
        lap = sum(_disk_potential(x + h * e)[0] + _disk_potential(x - h * e)[0] for e in np.eye(3)) \
            - 6 * _disk_potential(x)[0]
        assert abs(lap / h ** 2) < 1e-4
    far = np.array([[0.0, 0.0, 1e4]])
    assert abs(_disk_potential(far)[0] * 1e4 - 2.0 / math.pi) < 1e-6
    _, _, t4 = _golden()
    b, a, xr, sig = t4[0]
    def fd(dz):   # one-sided difference quotient of -du/dz on the top face
        return (1.0 - _disk_potential([[xr, 0.0, dz]])[0]) / dz
    dudn = 2.0 * fd(5e-5) - fd(1e-4)   # Richardson: the O(dz) term cancels
    assert abs(dudn - sig) < 1e-5, dudn
    assert abs(2.0 / (math.pi * math.sqrt(b * b - xr * xr)) - sig) < 1e-6


def test_thin_disk_distance_and_frame():
    g, _ = W.thin_disk()
    pts = np.array([[0.3, 0.4, 0.2], [3.0, 4.0, 1.0], [0.0, -2.0, -0.5]])
    d, nb = O.distance(g, pts)
    assert np.allclose(d, [0.2, math.hypot(4.0, 1.0), math.hypot(1.0, 0.5)], atol=1e-15)
    assert np.allclose(nb, [[0.3, 0.4, 0.0], [0.6, 0.8, 0.0], [0.0, -1.0, 0.0]], atol=1e-15)
    assert O.patch_frame(g, [-0.5, 0.0, 0.0], 0.4) is not None
    assert O.single_point(g, W.Dirichlet(W.DATA_CONSTANT, constant=1.0), [-0.5, 0, 0], 0.6, 4, 4, 1e-6,
                          U_in=np.zeros(16)) is None   # the ball's slice leaves the disk


def test_thin_disk_exact_hemisphere_values_and_walks():
    """Test 4: with the exact potential on the hemisphere the rule gives the
    analytic density (Sigma2' = 0 for constant data); walks that either reach the
    disk or leave the truncation sphere give Sigma1' within 4 standard errors."""
    g, d = W.thin_disk()
    _, _, t4 = _golden()
    b, a, xr, sig = t4[0]
    x = np.array([xr, 0.0, 0.0])
    pf = O.patch_frame(g, x, a)
    _, yg, _ = O.gamma_nodes(pf, 20, 20)
    r = O.single_point(g, d, x, a, 20, 20, 1e-6 * a, U_in=_disk_potential(yg.reshape(-1, 3), b))
    assert abs(r["sigma2"]) < 1e-15
    assert abs(r["q"] - sig) < 2e-4 * sig, r["q"]
    _, yg6, _ = O.gamma_nodes(pf, 6, 6)
    r0 = O.single_point(g, d, x, a, 6, 6, 1e-6 * a, U_in=_disk_potential(yg6.reshape(-1, 3), b))
    rw = O.single_point(g, d, x, a, 6, 6, 1e-6 * a, walks=300, patch=5, opts=O.wos_opts(eps=1e-5))
    assert rw["se"] > 0 and abs(rw["sigma1"] - r0["sigma1"]) <= 4 * rw["se"] + 1e-4
