"""Pins for the CNN oracle: finite differences, a closed form, and equivariance."""
import numpy as np

from oracle import cnn


def _problem(ny=7, nx=9, K=3, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((ny * nx, K)), rng.standard_normal((ny * nx, K)), (ny, nx)


def test_gradients_match_finite_differences():
    R, X, shape = _problem()
    p = cnn.init_params(C=4, seed=1, scale=0.5)
    L, g = cnn.loss_and_grad(p, R, X, shape)
    rng = np.random.default_rng(2)
    for key in p:
        for _ in range(4):
            idx = tuple(rng.integers(0, n) for n in p[key].shape)
            h = 1e-6
            q = {k: v.copy() for k, v in p.items()}
            q[key][idx] += h
            Lp, _ = cnn.loss_and_grad(q, R, X, shape)
            q[key][idx] -= 2 * h
            Lm, _ = cnn.loss_and_grad(q, R, X, shape)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[key][idx]) <= 1e-6 * max(1.0, abs(fd)), (key, idx, fd, g[key][idx])


def test_single_tap_filter_is_a_shift():
    """A filter with one unit tap shifts the image; zero padding fills the border."""
    ny, nx = 5, 6
    u = np.arange(ny * nx, dtype=float).reshape(1, ny, nx)
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 0, 2] = 1.0   # tap (dy, dx) = (0, 2): input at (y - 1, x + 1)
    y = cnn.conv(u, w, np.zeros(1))[0]
    for yy in range(ny):
        for xx in range(nx):
            ref = u[0, yy - 1, xx + 1] if (yy >= 1 and xx + 1 < nx) else 0.0
            assert y[yy, xx] == ref


def test_laplacian_filter_matches_the_stencil_matrix():
    """The 5-point filter equals the 2D Laplacian stencil matrix on the grid (x fastest)."""
    import workloads as wl

    k = 6
    A = wl.laplacian_2d(k)
    u = np.random.default_rng(0).standard_normal(k * k)
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 1, 1] = -4.0
    w[0, 0, 0, 1] = w[0, 0, 2, 1] = w[0, 0, 1, 0] = w[0, 0, 1, 2] = 1.0
    y = cnn.conv(u.reshape(1, k, k), w * (k + 1) ** 2, np.zeros(1)).reshape(-1)
    assert np.allclose(y, A @ u, rtol=1e-12, atol=1e-9)


def test_relu_network_is_positively_homogeneous_without_biases():
    p = cnn.init_params(C=4, seed=3)
    for b in ("b1", "b2", "b3"):
        p[b][:] = 0.0
    u = np.random.default_rng(4).standard_normal(30)
    y1, _ = cnn.forward(p, u, (5, 6))
    y2, _ = cnn.forward(p, 3.5 * u, (5, 6))
    assert np.allclose(y2, 3.5 * y1, rtol=1e-12, atol=1e-14)


def test_energy_loss_gradient_matches_finite_differences():
    import workloads as wl

    k = 7
    A = wl.laplacian_2d(k)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((k * k, 2))
    R = A @ X
    p = cnn.init_params(C=3, seed=2, scale=0.5)
    for jac in (False, True):
        L, g = cnn.energy_loss_and_grad(p, A, R, X, (k, k), jacobi=jac)
        for key in ("w1", "w2", "b2", "w3"):
            idx = tuple(rng.integers(0, n) for n in p[key].shape)
            h = 1e-6
            q = {kk: v.copy() for kk, v in p.items()}
            q[key][idx] += h
            Lp, _ = cnn.energy_loss_and_grad(q, A, R, X, (k, k), jacobi=jac)
            q[key][idx] -= 2 * h
            Lm, _ = cnn.energy_loss_and_grad(q, A, R, X, (k, k), jacobi=jac)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[key][idx]) <= 1e-6 * max(1.0, abs(fd)), (key, jac, fd, g[key][idx])
    # a zero network has loss exactly 1 (y = 0); with the Jacobi term, the loss of Jacobi scaling
    z = {kk: np.zeros_like(v) for kk, v in p.items()}
    L0, _ = cnn.energy_loss_and_grad(z, A, R, X, (k, k))
    assert abs(L0 - 1.0) <= 1e-12
    LJ, _ = cnn.energy_loss_and_grad(z, A, R, X, (k, k), jacobi=True)
    ref = 0.0
    for c in range(2):
        nr = np.linalg.norm(R[:, c])
        r, x = R[:, c] / nr, X[:, c] / nr
        d = r / A.diagonal() - x
        ref += float(d @ (-(A @ d))) / float(x @ (-(A @ x))) / 2
    assert abs(LJ - ref) <= 1e-12 * ref
