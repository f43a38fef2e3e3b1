"""Pins of the learned incomplete factor (oracle/learned_factor.py).

  * A network with a zero last layer gives the IC(0) factor exactly (the fallback).
  * On pairs that L0 L0^T solves exactly (r = L0 L0^T x) the loss at IC(0) is zero.
  * Finite differences confirm the gradients w.r.t. the factor values and the parameters.
  * A short training on the operator's own solve pairs lowers the loss and makes CG with
    P = (L L^T)^{-1} take fewer iterations than IC(0)-CG on that operator.
  * The channel conventions: output 1 scales the west entry, output 2 the south entry; the
    feature channels are centre, west, east, south, north, zero across the boundary.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as wl
from oracle import learned_factor as lf, pcg


def _operator(k, seed=1000):
    kappa = np.exp(1.5 * wl.gaussian_field(k, 2, seed=seed, corr_len=2.0))
    return sp.csr_matrix(-wl.var_coeff_diffusion(kappa))


def test_zero_last_layer_is_ic0():
    k = 12
    M = _operator(k)
    pat = lf.Pattern(M, k)
    p = lf.init_params(8, seed=1)
    y, _ = lf.forward(p, lf.stencil_features(M, k))
    assert np.array_equal(lf.factor_values(pat, y), pat.L0.data)


def test_loss_vanishes_on_pairs_exact_for_ic0():
    k = 10
    M = _operator(k)
    pat = lf.Pattern(M, k)
    X = np.random.default_rng(2).standard_normal((k * k, 5))
    R = pat.L0 @ (pat.L0.T @ X)
    loss, g = lf.loss_and_grad_values(pat, pat.L0.data.copy(), R, X)
    assert loss <= 1e-28 and np.max(np.abs(g)) <= 1e-12
    # and the loss of the exact factor of M on M's own pairs is not zero (IC(0) drops fill)
    loss_m, _ = lf.loss_and_grad_values(pat, pat.L0.data.copy(), M @ X, X)
    assert loss_m > 1e-6


def test_value_gradient_by_finite_differences():
    k = 8
    M = _operator(k)
    pat = lf.Pattern(M, k)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((k * k, 3))
    R = M @ X
    v = pat.L0.data * (1.0 + 0.05 * rng.standard_normal(pat.L0.data.shape))
    _, g = lf.loss_and_grad_values(pat, v, R, X)
    for i in rng.choice(v.size, 6, replace=False):
        h = 1e-6 * max(1.0, abs(v[i]))
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        fd = (lf.loss_and_grad_values(pat, vp, R, X)[0] - lf.loss_and_grad_values(pat, vm, R, X)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, g[i])


def test_parameter_gradient_by_finite_differences():
    k = 8
    M = _operator(k)
    pat = lf.Pattern(M, k)
    feats = lf.stencil_features(M, k)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((k * k, 3))
    R = M @ X
    p = lf.init_params(4, seed=5)
    p["w3"] = 0.05 * rng.standard_normal(p["w3"].shape)  # so that every layer receives gradient
    p["b1"] = 0.05 * rng.standard_normal(p["b1"].shape)
    _, g = lf.loss_and_grad(p, pat, feats, R, X)
    for key in ("w1", "b1", "w2", "w3", "b3"):
        flat = p[key].reshape(-1)
        for i in rng.choice(flat.size, 2, replace=False):
            old = flat[i]
            h = 1e-6
            flat[i] = old + h
            lp = lf.loss_and_grad(p, pat, feats, R, X)[0]
            flat[i] = old - h
            lm = lf.loss_and_grad(p, pat, feats, R, X)[0]
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            gi = g[key].reshape(-1)[i]
            assert abs(fd - gi) <= 1e-4 * max(1e-3, abs(fd)), (key, i, fd, gi)


def test_short_training_beats_ic0():
    k = 32
    M = _operator(k)
    n = k * k
    pat = lf.Pattern(M, k)
    feats = lf.stencil_features(M, k)
    rng = np.random.default_rng(0)
    R = rng.standard_normal((n, 16))
    X = spla.splu(sp.csc_matrix(M)).solve(R)
    p = lf.init_params(16, seed=0)
    mom = {a: np.zeros_like(v) for a, v in p.items()}
    vel = {a: np.zeros_like(v) for a, v in p.items()}
    first = None
    iters, lr = 300, 3e-3
    for it in range(1, iters + 1):
        idx = rng.choice(R.shape[1], 8, replace=False)
        loss, g = lf.loss_and_grad(p, pat, feats, R[:, idx], X[:, idx])
        first = loss if first is None else first
        for a in p:  # Adam
            mom[a] = 0.9 * mom[a] + 0.1 * g[a]
            vel[a] = 0.999 * vel[a] + 0.001 * g[a] ** 2
            p[a] -= lr * (mom[a] / (1 - 0.9**it)) / (np.sqrt(vel[a] / (1 - 0.999**it)) + 1e-12)
    y, _ = lf.forward(p, feats)
    L = lf.build_L(pat, lf.factor_values(pat, y))
    final, _ = lf.loss_and_grad_values(pat, lf.factor_values(pat, y), R, X)
    assert final < 0.1 * first
    b = wl.rhs(n, 1, seed=100)[:, 0]
    it_ic0 = pcg.pcg(M, b, prec=pcg.ic0_prec(pat.L0), tol=1e-8).iterations
    it_net = pcg.pcg(M, b, prec=pcg.ic0_prec(L), tol=1e-8).iterations
    assert it_net < it_ic0, (it_net, it_ic0)


def test_channel_conventions():
    """Output channel 1 scales the west entry L_{i,i-1}, channel 2 the south entry L_{i,i-k};
    feature channels are (centre, west, east, south, north), zero across the boundary."""
    k = 6
    M = _operator(k)
    pat = lf.Pattern(M, k)
    i = 3 * k + 2  # an interior node
    for ch, col in ((1, i - 1), (2, i - k), (0, i)):
        y = np.zeros((3, k, k))
        y[ch].reshape(-1)[i] = 0.5
        changed = lf.factor_values(pat, y) != pat.L0.data
        assert np.array_equal(np.flatnonzero(changed), np.flatnonzero((pat.rows == i) & (pat.cols == col)))
    f = lf.stencil_features(M, k).reshape(5, -1)
    x, yy = np.arange(k * k) % k, np.arange(k * k) // k
    assert np.all(f[1][x == 0] == 0) and np.all(f[1][x > 0] < 0)          # west
    assert np.all(f[2][x == k - 1] == 0) and np.all(f[2][x < k - 1] < 0)  # east
    assert np.all(f[3][yy == 0] == 0) and np.all(f[4][yy == k - 1] == 0)  # south, north
    assert np.allclose(f[1][1:], M.diagonal()[1:] ** -1 * np.asarray(M[np.arange(1, k * k), np.arange(k * k - 1)]).ravel()
                       * (x[1:] > 0))
