"""Pins of the truncated-Neumann IC(0) preconditioner and its learned values (oracle/neumann_ic).

What fixes each part, independently of the functions under test:
  * B_q with q = 0 is D^{-1}; B_q L = I - T^{q+1} with L from oracle/pcg.ic0 applied by scipy and
    T^{q+1} formed as a sparse matrix power (telescoping sum of the Neumann series);
  * for large q, P_q r is the exact (L L^T)^{-1} r by two triangular solves (T is nilpotent);
  * B_q^T is the transpose of B_q and P_q is symmetric positive definite (dense, tiny grid);
  * the gradients w.r.t. the factor values and the network's parameters equal central
    finite differences of the loss;
  * a zero last layer reproduces IC(0) exactly;
  * training on the method's first solve pair (C iid N(0,1), x = M^{-1} C) lowers the loss and
    the conjugate-gradient iterations below IC(0) with the same truncation (the gain the GPU
    test then measures), and the trained preconditioner still converges where Jacobi does;
  * planted mistakes (a wrong sign of T, a dropped gradient term) fail these pins.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as wl
from oracle import learned_factor as lf
from oracle import neumann_ic as ni
from oracle import pcg


def _op(k, seed=3, corr=2.0, sigma=1.5):
    kap = np.exp(sigma * wl.gaussian_field(k, 2, seed=seed, corr_len=corr))
    return sp.csr_matrix(-wl.var_coeff_diffusion(kap))


def _t_matrix(L):
    L = sp.csr_matrix(L)
    d = L.diagonal()
    N = L - sp.diags(d)
    return sp.csr_matrix(-sp.diags(1.0 / d) @ N), d


@pytest.mark.parametrize("q", [0, 1, 3, 5])
def test_telescoping_identity(q):
    k = 7
    M = _op(k)
    L = pcg.ic0(M)
    d, lw, ls = ni.factor_arrays(L, k)
    T, _ = _t_matrix(L)
    r = np.random.default_rng(q).standard_normal(k * k)
    lhs = ni.apply_B(d, lw, ls, k, q, L @ r)[:, 0]
    Tq = sp.identity(k * k, format="csr")
    for _ in range(q + 1):
        Tq = Tq @ T
    assert np.allclose(lhs, r - Tq @ r, rtol=0, atol=1e-12 * np.linalg.norm(r))
    if q == 0:
        assert np.allclose(ni.apply_B(d, lw, ls, k, 0, r)[:, 0], r / d)


def test_large_q_is_the_exact_ic0_solve():
    k = 6
    M = _op(k, seed=5)
    L = pcg.ic0(M)
    d, lw, ls = ni.factor_arrays(L, k)
    r = np.random.default_rng(2).standard_normal(k * k)
    ex = pcg.ic0_prec(L)(r)
    got = ni.apply_P(d, lw, ls, k, 2 * k * k, r)[:, 0]
    assert np.allclose(got, ex, rtol=1e-12, atol=1e-12 * np.linalg.norm(ex))


def test_transpose_and_definiteness():
    k = 6
    M = _op(k, seed=7)
    d, lw, ls = ni.ic0_arrays(M, k)
    n = k * k
    I = np.eye(n)
    B = ni.apply_B(d, lw, ls, k, 3, I)
    Bt = ni.apply_Bt(d, lw, ls, k, 3, I)
    assert np.allclose(Bt, B.T, atol=1e-14 * np.abs(B).max())
    assert np.allclose(np.tril(B), B)
    assert np.allclose(np.diag(B), 1.0 / d)
    P = ni.apply_P(d, lw, ls, k, 3, I)
    assert np.allclose(P, P.T, atol=1e-13 * np.abs(P).max())
    assert np.linalg.eigvalsh(P).min() > 0


def _fd_values(fun, arrs, grads, rng, h=1e-6):
    for idx in range(3):
        v = rng.standard_normal(arrs[idx].shape) * (arrs[idx] != 0)
        up = list(arrs)
        dn = list(arrs)
        up[idx] = arrs[idx] + h * v
        dn[idx] = arrs[idx] - h * v
        fd = (fun(*up) - fun(*dn)) / (2 * h)
        an = float(grads[idx] @ v)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-8), (idx, fd, an)


def test_value_gradient_matches_finite_differences():
    k = 8
    M = _op(k)
    d, lw, ls = ni.ic0_arrays(M, k)
    rng = np.random.default_rng(0)
    R = rng.standard_normal((k * k, 2))
    X = spla.spsolve(sp.csc_matrix(M), R)
    for q in (1, 3):
        loss, g = ni.energy_loss_and_grad_values(d, lw, ls, k, q, M, R, X)
        assert loss == pytest.approx(ni.energy_loss(d, lw, ls, k, q, M, R, X), rel=1e-14)
        _fd_values(lambda a, b, c: ni.energy_loss(a, b, c, k, q, M, R, X), (d, lw, ls), g, rng)


def test_network_gradient_matches_finite_differences():
    k = 8
    M = _op(k)
    d0, lw0, ls0 = ni.ic0_arrays(M, k)
    feats = lf.stencil_features(M, k)
    rng = np.random.default_rng(1)
    p = lf.init_params(16, 0, 0.3)
    p["w3"] = rng.standard_normal(p["w3"].shape) * 0.05
    p["b3"] = rng.standard_normal(3) * 0.01
    R = rng.standard_normal((k * k, 2))
    X = spla.spsolve(sp.csc_matrix(M), R)
    loss, g = ni.net_loss_and_grad(p, feats, d0, lw0, ls0, k, 3, M, R, X)

    def L(pp):
        return ni.energy_loss(*ni.net_values(pp, feats, d0, lw0, ls0)[:3], k, 3, M, R, X)

    h = 1e-6
    for key in p:
        v = rng.standard_normal(p[key].shape)
        up = {a: b.copy() for a, b in p.items()}
        dn = {a: b.copy() for a, b in p.items()}
        up[key] = p[key] + h * v
        dn[key] = p[key] - h * v
        fd = (L(up) - L(dn)) / (2 * h)
        an = float(np.sum(g[key] * v))
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-6), (key, fd, an)


def test_zero_last_layer_is_ic0():
    k = 9
    M = _op(k)
    d0, lw0, ls0 = ni.ic0_arrays(M, k)
    p = lf.init_params(16, 2, 0.1)
    d, lw, ls, _ = ni.net_values(p, lf.stencil_features(M, k), d0, lw0, ls0)
    assert np.array_equal(d, d0) and np.array_equal(lw, lw0) and np.array_equal(ls, ls0)


def test_training_on_the_first_solve_pair_beats_ic0():
    k = 64
    M = _op(k, seed=1000, corr=16.0)
    n = k * k
    d0, lw0, ls0 = ni.ic0_arrays(M, k)
    feats = lf.stencil_features(M, k)
    C = wl.rhs(n, 2, 0)
    X = spla.splu(sp.csc_matrix(M)).solve(C)
    p, losses = ni.train(lf.init_params(16, 0, 0.1), feats, d0, lw0, ls0, k, 3, M, C, X, 150, 3e-3)
    assert losses[-1] < 0.9 * losses[0]
    d, lw, ls, _ = ni.net_values(p, feats, d0, lw0, ls0)
    b = np.random.default_rng(5).standard_normal(n)
    it_ic = pcg.pcg(M, b, ni.prec(d0, lw0, ls0, k, 3), tol=1e-8).iterations
    res = pcg.pcg(M, b, ni.prec(d, lw, ls, k, 3), tol=1e-8)
    it_jac = pcg.pcg(M, b, pcg.jacobi_prec(M), tol=1e-8, maxit=50000).iterations
    assert res.converged and np.linalg.norm(M @ res.x - b) <= 1e-7 * np.linalg.norm(b)
    print("CG iterations: Jacobi", it_jac, "IC(0) q=3", it_ic, "learned q=3", res.iterations)
    assert res.iterations <= 0.9 * it_ic < it_jac


def test_planted_mistakes_fail(monkeypatch):
    k = 7
    M = _op(k)
    L = pcg.ic0(M)
    d, lw, ls = ni.factor_arrays(L, k)
    T, _ = _t_matrix(L)
    r = np.random.default_rng(9).standard_normal(k * k)
    q = 2
    Tq = T @ T @ T
    good = np.allclose(ni.apply_B(d, lw, ls, k, q, L @ r)[:, 0], r - Tq @ r, atol=1e-12 * np.linalg.norm(r))
    assert good
    # a wrong sign of T
    monkeypatch.setattr(ni, "t_apply", lambda d_, w_, s_, nx, V: ni.n_apply(w_, s_, nx, V) / d_[:, None])
    bad = np.allclose(ni.apply_B(d, lw, ls, k, q, L @ r)[:, 0], r - Tq @ r, atol=1e-12 * np.linalg.norm(r))
    assert not bad
    monkeypatch.undo()
    # the trailing-D^{-1} term of the gradient dropped
    rng = np.random.default_rng(4)
    R = rng.standard_normal((k * k, 1))
    X = spla.spsolve(sp.csc_matrix(M), R)[:, None]
    loss, (gd, gw, gs) = ni.energy_loss_and_grad_values(d, lw, ls, k, 2, M, R, X)
    orig = ni.bilinear_grad

    def dropped(d_, w_, s_, nx, q_, A_, C_):
        # adds back the t = 0 trailing-D^{-1} term, i.e. drops it
        g = orig(d_, w_, s_, nx, q_, A_, C_)
        return (g[0] + np.sum(ni._col(A_) * ni._col(C_), axis=1) / d_**2, g[1], g[2])

    monkeypatch.setattr(ni, "bilinear_grad", dropped)
    _, (gd2, _, _) = ni.energy_loss_and_grad_values(d, lw, ls, k, 2, M, R, X)
    v = rng.standard_normal(k * k)
    h = 1e-6
    fd = (ni.energy_loss(d + h * v, lw, ls, k, 2, M, R, X) - ni.energy_loss(d - h * v, lw, ls, k, 2, M, R, X)) / (2 * h)
    assert abs(fd - gd @ v) <= 1e-6 * abs(fd)
    assert abs(fd - gd2 @ v) > 1e-3 * abs(fd)
