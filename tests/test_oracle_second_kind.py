"""Oracle pins for the second-kind local BIE on flat patches (Eq. bw53-bw59):
the kernel d2G/dn_x dn_y against finite differences of the Green's function,
the vanishing double layer on a plane through the ball centre, the constant
solution, and the Neumann data with the exact solution on the hemisphere."""
import numpy as np

import oracle as O
import workloads as W


def test_normal_normal_kernel_matches_finite_differences():
    rng = np.random.default_rng(0)
    for a in (0.3, 1.0):
        for _ in range(4):
            X = rng.normal(size=3) * 0.25 * a
            Y = rng.normal(size=3) * 0.35 * a
            nx = rng.normal(size=3); nx /= np.linalg.norm(nx)
            ny = rng.normal(size=3); ny /= np.linalg.norm(ny)
            h = 1e-4 * a
            G = lambda P, Q: O.green(a, P, Q)
            fd = (G(X + h * nx, Y + h * ny) - G(X + h * nx, Y - h * ny) - G(X - h * nx, Y + h * ny)
                  + G(X - h * nx, Y - h * ny)) / (4 * h * h)
            k = O.green_dnn(a, X, nx, Y, ny)
            assert abs(k - fd) <= 1e-5 * max(1.0, abs(k)), (k, fd)


def test_double_layer_vanishes_in_the_plane_through_the_centre():
    rng = np.random.default_rng(1)
    n = np.array([0.0, 0.0, 1.0])
    for _ in range(5):
        X = np.r_[rng.normal(size=2) * 0.3, 0.0]
        Y = np.r_[rng.normal(size=2) * 0.3, 0.0]
        # dG/dn_x (x, y) = n . grad_X G(X, Y) = n . grad_y G(Y, X) by symmetry
        assert abs(np.dot(O.green_grad_y(0.5, Y, X), n)) < 1e-12


def test_constant_solution_gives_zero():
    wl = W.cube_single_patch()
    pf = O.patch_frame(wl.geometry, wl.batch.centers[0], 0.1)
    const = W.Dirichlet(W.DATA_CONSTANT, constant=3.0)
    q = O.second_kind_flat(pf, const, 8, 16, 4, 8, np.full(128, 3.0))
    assert np.max(np.abs(q)) < 1e-10


def test_exact_hemisphere_values_give_the_neumann_data():
    """Point-source data on the unit-cube face: with the exact solution at the
    hemisphere nodes the rows give the exact Neumann data inside r < 0.7a to
    1e-3 (16 x 32 nodes) and 5e-4 (32 x 64); the rim rows carry the error of
    the hemisphere rule next to the near-singular kernel."""
    wl = W.cube_single_patch()
    pf = O.patch_frame(wl.geometry, wl.batch.centers[0], 0.1)
    pan = O.panels(pf, 8, 8)
    qe = O.neumann_exact(wl.data, pan["x"], pan["normal"])
    inner = np.linalg.norm(pan["Xloc"][:, :2], axis=1) < 0.07
    for nt, bound in ((16, 1e-3), (32, 5e-4)):
        _, yg, _ = O.gamma_nodes(pf, nt, 2 * nt)
        U = O.dirichlet(wl.data, yg.reshape(-1, 3))
        q = O.second_kind_flat(pf, wl.data, nt, 2 * nt, 8, 8, U, ng2=20)
        rel = np.abs(q - qe) / np.abs(qe)
        assert rel[inner].max() <= bound, (nt, rel[inner].max())


# ----------------------------------------------------------------- any patch (cap or disk)
# or_second_kind: (1/2 I - D) q = b with D_ij = int_{panel j} dG/dn_x(x_i, y) ds_y and the
# finite part regularised by the harmonic function l_i = g(x_i) + grad_S g(x_i).(y - x_i).

def _ball_cap(i=3, a=0.1):
    wl = W.unit_ball(n_patches=20)
    return wl, O.patch_frame(wl.geometry, wl.batch.centers[i], a)


def test_general_constant_solution_gives_zero():
    _, pf = _ball_cap()
    const = W.Dirichlet(W.DATA_CONSTANT, constant=2.0)
    q = O.second_kind(pf, const, 16, 32, 4, 8, np.full(16 * 32, 2.0))
    assert np.max(np.abs(q)) < 1e-12


def test_general_rows_agree_with_flat_rows_on_a_disk():
    """Two regularisations of the linear Taylor term (the exact rim integral of
    the flat rows, the identity for the harmonic l_i here) give the same inner
    rows."""
    wc = W.cube_single_patch()
    pd = O.patch_frame(wc.geometry, wc.batch.centers[0], 0.1)
    _, yg, _ = O.gamma_nodes(pd, 16, 32)
    U = O.dirichlet(wc.data, yg.reshape(-1, 3))
    pan = O.panels(pd, 8, 8)
    inner = np.linalg.norm(pan["Xloc"][:, :2], axis=1) < 0.07
    qf = O.second_kind_flat(pd, wc.data, 16, 32, 8, 8, U, ng2=48)
    qg = O.second_kind(pd, wc.data, 16, 32, 8, 8, U, rtol=1e-10)
    assert np.max(np.abs(qg - qf)[inner]) <= 5e-4 * np.max(np.abs(qf))


def test_cap_exact_hemisphere_values_give_the_neumann_data():
    """Harmonic data r^l Y_lm on the unit ball (exact Neumann data
    sum l c_lm Y_lm): with the exact solution at the hemisphere nodes the cap
    rows match it inside r < 0.7a to 1e-3 of max|q|, and the system is well
    conditioned (cond ~ 1)."""
    wl, pf = _ball_cap()
    nr, ns, nt, nph = 4, 8, 16, 32
    _, yg, _ = O.gamma_nodes(pf, nt, nph)
    U = O.dirichlet(wl.data, yg.reshape(-1, 3))
    pan = O.panels(pf, nr, ns)
    qe = O.neumann_exact(wl.data, pan["x"], pan["normal"])
    q, A, b = O.second_kind(pf, wl.data, nt, nph, nr, ns, U, want_system=True)
    inner = np.linalg.norm(pan["Xloc"][:, :2], axis=1) < 0.07
    scale = np.max(np.abs(qe))
    assert np.max(np.abs(q - qe)[inner]) <= 1e-3 * scale
    assert np.max(np.abs(q - qe)) <= 0.1 * scale
    assert np.linalg.cond(A) < 1.2



def _cap_point(pf, u, v):
    R = pf.R
    return np.array([R * np.sin(u) * np.cos(v), R * np.sin(u) * np.sin(v), -2 * R * np.sin(0.5 * u) ** 2])


def test_double_layer_row_sums_match_a_geodesic_polar_rule():
    """sum_j D_ij = int_S dG/dn_x(x_i, y) ds_y (the panels' constant basis sums
    to one).  Brute force: geodesic polar coordinates (sigma, phi) about x_i on
    the sphere, the cap's edge at sigma_max(phi) from spherical trigonometry,
    48 x 48 Gauss points; the integrand is bounded there (the 1/r of dG/dn_x
    on a sphere against the Jacobian R^2 sin sigma)."""
    wl, pf = _ball_cap(a=0.15)
    nr, ns = 2, 4
    q, A, b = O.second_kind(pf, wl.data, 4, 8, nr, ns, np.zeros(32), want_system=True)
    D = 0.5 * np.eye(nr * ns) - A
    pan = O.panels(pf, nr, ns)
    R, a = pf.R, pf.a
    o = np.array([0.0, 0.0, -R])                        # sphere centre, local frame
    x, w = np.polynomial.legendre.leggauss(48)
    for i in range(nr * ns):
        X = pan["Xloc"][i]
        p = (X - o) / R
        nx = p                                         # outward unit normal at X
        e1 = np.cross(p, [0.0, 1.0, 0.0]); e1 /= np.linalg.norm(e1)
        e2 = np.cross(p, e1)
        tot = 0.0
        for phi, wp in zip(np.pi * (x + 1), np.pi * w):
            d = np.cos(phi) * e1 + np.sin(phi) * e2
            A0, B0 = p[2], d[2]
            C0 = np.hypot(A0, B0)
            smax = np.arctan2(B0, A0) + np.arccos(np.cos(pf.umax) / C0)
            for sg, ws in zip(0.5 * smax * (x + 1), 0.5 * smax * w):
                Y = o + R * (np.cos(sg) * p + np.sin(sg) * d)
                dnx = float(np.dot(O.green_grad_y(a, Y, X), nx))
                tot += wp * ws * dnx * R * R * np.sin(sg)
        assert abs(D[i].sum() - tot) <= 1e-9 * max(1.0, abs(tot)), (i, D[i].sum(), tot)


def test_self_panel_rule_has_converged():
    """The second kind's self-panel integrals (Duffy triangles, a fixed Gauss
    rule of order m per direction): the integrand is smooth in the Duffy
    variables, so the orders 12 ... 24 must agree to the rounding floor.  q at
    order 20 (the default) is within 2e-11 (relative L2) of q at 12, 16 and 24,
    on a unit-ball cap and on the R = 3 sphere seen from outside."""
    cases = []
    wl, pf = _ball_cap()
    cases.append((wl, pf, lambda y: O.dirichlet(wl.data, y)))
    we = W.sphere_exterior(n_patches=2, walks=2)
    pe = O.patch_frame(we.geometry, we.batch.centers[0], 1.0)
    cases.append((we, pe, lambda y: 3.0 / np.linalg.norm(y, axis=1)))
    assert O.set_sk_self_order(20) == 20
    try:
        for wl_, pf_, u in cases:
            _, yg, _ = O.gamma_nodes(pf_, 16, 32)
            U = u(yg.reshape(-1, 3))
            qs = {}
            for m in (12, 16, 20, 24):
                O.set_sk_self_order(m)
                qs[m] = O.second_kind(pf_, wl_.data, 16, 32, 4, 8, U)
            ref = qs[20]
            for m in (12, 16, 24):
                assert np.linalg.norm(qs[m] - ref) <= 2e-11 * np.linalg.norm(ref), m
    finally:
        O.set_sk_self_order(20)
