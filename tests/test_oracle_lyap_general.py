"""Pins of the generalised Lyapunov oracle (oracle/lyap_general.py): A X E + E X A + C C^T = 0
with a finite-element mass matrix E.

  * E = I gives exactly the standard solve (same history, same m).
  * The factored X agrees with a dense solve of the original equation written out with
    Kronecker products, (E (x) A + A (x) E) vec(X) = -vec(C C^T), which does not use the
    Cholesky transformation.
  * The original residual A X E + E X A + C C^T equals L R~ L^T, R~ the residual of the
    transformed equation, and is small at convergence.
  * The transformed operator is symmetric negative definite, so Alg. 1-3 apply.
"""
import numpy as np
import scipy.sparse as sp

import workloads as wl
from oracle import lyap, lyap_general as lg


def test_identity_mass_matrix_is_the_standard_equation():
    A = wl.laplacian_2d(10)
    C = wl.rhs(100, 2, seed=3)
    rg = lg.solve(A, sp.identity(100, format="csr"), C, tol=1e-9, maxit=200)
    rs = lyap.solve(A.toarray(), C, tol=1e-9, maxit=200)
    assert rg.inner.m == rs.m
    assert np.allclose(rg.inner.history, rs.history, rtol=1e-10, atol=0)


def test_factor_matches_kronecker_solve():
    k = 7
    A, E = wl.fe_mass_stiffness_2d(k)
    n = k * k
    C = wl.rhs(n, 2, seed=4)
    res = lg.solve(A, E, C, tol=1e-11, maxit=300)
    assert res.inner.converged
    Z, _ = lg.factor(res, trunc_eps=1e-14)
    X = Z @ Z.T
    Ad, Ed = A.toarray(), E.toarray()
    K = np.kron(Ed, Ad) + np.kron(Ad, Ed)
    X_ref = np.linalg.solve(K, -(C @ C.T).reshape(-1, order="F")).reshape(n, n, order="F")
    assert np.linalg.norm(X - X_ref) <= 1e-8 * np.linalg.norm(X_ref)


def test_residual_maps_by_the_cholesky_factor():
    k = 9
    A, E = wl.fe_mass_stiffness_2d(k, kappa=np.exp(wl.gaussian_field(k + 1, 2, seed=2)))
    C = wl.rhs(k * k, 2, seed=5)
    res = lg.solve(A, E, C, tol=1e-10, maxit=300)
    assert res.inner.converged
    assert np.max(np.linalg.eigvalsh(res.At)) < 0.0
    Z, _ = lg.factor(res, trunc_eps=1e-14)
    X = Z @ Z.T
    Ad, Ed = A.toarray(), E.toarray()
    R = Ad @ X @ Ed + Ed @ X @ Ad + C @ C.T
    Xt = res.L.T @ X @ res.L
    Rt = res.At @ Xt + Xt @ res.At + res.Ct @ res.Ct.T
    assert np.linalg.norm(R - res.L @ Rt @ res.L.T) <= 1e-10 * np.linalg.norm(C @ C.T)
    assert np.linalg.norm(R) <= 1e-8 * np.linalg.norm(C @ C.T)
