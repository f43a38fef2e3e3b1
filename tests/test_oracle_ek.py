"""Pins for the FP64 extended Krylov oracle (Sec. 4), independent of its own formulas."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import ek, explicit
from oracle import lyap as olyap


@pytest.fixture(scope="module")
def small():
    A = wl.laplacian_2d(12)
    C = wl.rhs(A.shape[0], 2, 4)
    return A, C, ek.solve(A, C, tol=1e-11, maxit=25)


def test_basis_is_orthonormal(small):
    A, C, r = small
    V = np.hstack(r.log.basis[: r.m + 1])
    assert np.linalg.norm(V.T @ V - np.eye(V.shape[1])) <= 1e-10


def test_older_coefficients_vanish_in_early_steps():
    """Sec. 4's three-term recurrence: W's components along blocks older than V_{j-1} are zero
    in exact arithmetic (they are at rounding level while little rounding has built up)."""
    A = wl.laplacian_2d(30)
    C = wl.rhs(900, 2, 4)
    inv = ek.factor_A(A)
    log = ek.start(A, C, inv)
    for j in range(1, 5):
        coefs = []
        log.basis.append(ek.step(A, inv, log.basis, coefs))
        scale = max(coefs)
        assert all(c <= 1e-9 * scale for c in coefs[:-2]), (j, coefs)
        assert coefs[-1] > 1e-3 * scale


def test_projected_matrix_is_block_tridiagonal(small):
    """V^T A V vanishes outside the block tridiagonal band, and A V_m = V_{m+1} [T_m; tau E_m^T]."""
    A, C, r = small
    S = 2 * r.log.s
    V = np.hstack(r.log.basis[: r.m + 1])
    T = V.T @ (A @ V)
    scale = np.abs(T).max()
    for i in range(r.m + 1):
        for j in range(r.m + 1):
            if abs(i - j) > 1:
                assert np.abs(T[i * S:(i + 1) * S, j * S:(j + 1) * S]).max() <= 1e-9 * scale
    Vm = V[:, : S * r.m]
    lhs = A @ Vm
    rhs = V @ T[:, : S * r.m]
    assert np.linalg.norm(lhs - rhs) <= 1e-9 * np.linalg.norm(lhs)


def test_cheap_residual_equals_reduced_bartels_stewart(small):
    """Prop. 3.1 on the extended T_m equals sqrt(2) ||Y E_m tau^T|| with Y from scipy's solver."""
    A, C, r = small
    S = 2 * r.log.s
    for m in (2, 5, r.m):
        ab = ek.band_T(r.log, m)
        N = S * m
        T = np.zeros((N, N))
        for d in range(S + 1):
            idx = np.arange(N - d)
            T[idx + d, idx] = ab[d, : N - d]
            T[idx, idx + d] = ab[d, : N - d]
        G = np.zeros((N, r.log.s))
        G[:S] = r.log.gamma[:, : r.log.s]
        Y = sla.solve_continuous_lyapunov(T, -G @ G.T)
        ref = np.sqrt(2.0) * np.linalg.norm(Y[:, -S:] @ r.log.tau_next[m - 1].T) / r.log.beta**2
        assert abs(ek.residual_at(r.log, m) - ref) <= 1e-10 * max(ref, 1e-14) + 1e-15


def test_cheap_residual_equals_explicit_residual():
    A = wl.laplacian_2d(9)
    C = wl.rhs(81, 1, 3)
    r = ek.solve(A, C, tol=0.0, maxit=6)
    for m in (2, 4, 6):
        sub = ek.EKResult(r.log, r.history[:m], m, False)
        Z, _ = ek.factor(sub, trunc_eps=0.0)
        X = Z @ Z.T
        R = A @ X + X @ A + C @ C.T
        assert abs(np.linalg.norm(R) / r.log.beta**2 - r.history[m - 1]) <= 1e-9 * r.history[m - 1] + 1e-13


def test_first_block_spans_C_and_Ainv_C(small):
    A, C, r = small
    V1 = r.log.basis[0]
    s = r.log.s
    assert np.linalg.norm(V1 @ r.log.gamma[:, :s] - C) <= 1e-12 * np.linalg.norm(C)
    sol = np.linalg.solve(A.toarray(), C)
    assert np.linalg.norm(V1 @ (V1.T @ sol) - sol) <= 1e-10 * np.linalg.norm(sol)


def test_extended_space_needs_fewer_iterations_than_standard():
    """On a Laplacian the extended space reaches the tolerance in far fewer (and smaller)
    iterations than the standard block Krylov space (Sec. 6 reports the same trend)."""
    A = wl.laplacian_2d(40)
    C = wl.rhs(A.shape[0], 1, 1)
    r = ek.solve(A, C, tol=1e-8, maxit=200)
    std = olyap.solve(A, C, tol=1e-8, maxit=1000)
    assert r.converged and std.converged
    assert 2 * r.m < std.m


def test_factor_solves_the_equation(small):
    """The untruncated factor reproduces the history's last value as an explicit residual
    (truncation at eps would add up to 2 ||A|| eps on top)."""
    A, C, r = small
    Z, _ = ek.factor(r, trunc_eps=0.0)
    rel = explicit.lyap_lowrank(A, Z, C) / r.log.beta**2
    assert abs(rel - r.history[-1]) <= 1e-6 * r.history[-1] + 1e-13


def test_planted_mistake_in_gamma_is_caught(small):
    """Using the full gamma (including the A^{-1} C part) as right-hand side changes the
    residual far beyond the 1e-10 tolerance of the Bartels-Stewart pin above, which therefore
    catches it: the reduced right-hand side is E_1 gamma_1 gamma_1^T E_1^T only."""
    A, C, r = small
    S = 2 * r.log.s
    lam, Q = sla.eig_banded(ek.band_T(r.log, 3), lower=True)
    good = olyap.cheap_residual(lam, Q, r.log.gamma1, r.log.tau_next[2], S)
    bad = olyap.cheap_residual(lam, Q, r.log.gamma, r.log.tau_next[2], S)
    assert abs(good - bad) > 1e-7 * good
