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
    rg = lg.solve(A, sp.identity(100, format="csr"), C, tol=1e-9, maxit=200, reorth=False)
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


def test_full_reorthogonalisation_keeps_the_basis_orthonormal_and_the_coefficients():
    """The default step (Gram-Schmidt against every stored block) keeps V~ orthonormal to rounding
    where the plain step of Alg. 2 loses it, and while the plain basis is still orthonormal the
    two give the same tau coefficients and history."""
    k = 14
    A, E = wl.fe_mass_stiffness_2d(k)
    C = wl.rhs(k * k, 2, seed=6)
    full = lg.solve(A, E, C, tol=0.0, maxit=60)
    plain = lg.solve(A, E, C, tol=0.0, maxit=60, reorth=False)
    Vf = np.hstack(full.inner.log.basis[:60])
    Vp = np.hstack(plain.inner.log.basis[:60])
    I = np.eye(Vf.shape[1])
    assert np.linalg.norm(Vf.T @ Vf - I) <= 1e-12
    assert np.linalg.norm(Vp.T @ Vp - I) >= 1e-6  # the plain recurrence has lost orthogonality
    # early on both are orthonormal to rounding and agree
    for j in range(8):
        assert np.allclose(full.inner.log.tau_diag[j], plain.inner.log.tau_diag[j], rtol=0, atol=1e-9 * full.inner.log.beta)
    assert np.allclose(full.inner.history[:8], plain.inner.history[:8], rtol=1e-9, atol=0)
    # and the full-reorthogonalisation T_m is V~^T A~ V~ (the Galerkin projection), block by block
    T = lyap.dense_T(full.inner.log, 40)
    V40 = np.hstack(full.inner.log.basis[:40])
    assert np.linalg.norm(T - V40.T @ full.At @ V40) <= 1e-10 * np.linalg.norm(full.At, 2)
