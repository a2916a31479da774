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
