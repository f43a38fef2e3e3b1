"""Pins for the FP64 Sylvester oracle (Sec. 5.1, Alg. 4, eq. 5.5)."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import explicit, lyap, sylvester


@pytest.fixture(scope="module")
def sylv_problem():
    n1, n2, s = 80, 55, 2
    A = wl.random_snd_dense(n1, seed=1, lam_min=1.0, lam_max=200.0)
    B = wl.random_snd_dense(n2, seed=2, lam_min=0.5, lam_max=50.0)
    C1 = wl.rhs(n1, s, 3)
    C2 = wl.rhs(n2, s, 4)
    res = sylvester.solve(A, B, C1, C2, tol=0.0, maxit=10, keep_basis=True)
    return A, B, C1, C2, res


def _reduced_bs(res, m):
    s = res.logA.s
    T = lyap.dense_T(res.logA, m)
    J = lyap.dense_T(res.logB, m)
    E1 = np.zeros((s * m, s))
    E1[:s] = np.eye(s)
    rhs = -(E1 @ res.logA.gamma) @ (E1 @ res.logB.gamma).T
    Y = sla.solve_sylvester(T, J, rhs)
    tau = res.logA.tau_next[m - 1]
    iota = res.logB.tau_next[m - 1]
    r2 = np.linalg.norm(tau @ Y[-s:, :]) ** 2 + np.linalg.norm(Y[:, -s:] @ iota.T) ** 2
    return np.sqrt(r2), Y


def test_cheap_equals_reduced_bartels_stewart(sylv_problem):
    """eq. (5.5) with Y from scipy's Bartels-Stewart Sylvester solver."""
    *_, res = sylv_problem
    beta2 = res.logA.beta * res.logB.beta
    for m in range(1, res.m + 1):
        ref, _ = _reduced_bs(res, m)
        assert abs(res.history[m - 1] * beta2 - ref) <= 1e-10 * ref


def test_cheap_equals_explicit_residual(sylv_problem):
    A, B, C1, C2, res = sylv_problem
    beta2 = res.logA.beta * res.logB.beta
    for m in (1, 3, 6, 10):
        _, Y = _reduced_bs(res, m)
        Vm = np.hstack(res.logA.basis[:m])
        Um = np.hstack(res.logB.basis[:m])
        X = Vm @ Y @ Um.T
        R = A @ X + X @ B + C1 @ C2.T
        assert abs(np.linalg.norm(R) / beta2 - res.history[m - 1]) <= 1e-9 * res.history[m - 1]
        assert np.linalg.norm(Vm.T @ R @ Um) <= 1e-10 * np.linalg.norm(C1 @ C2.T)


def test_printed_pairing_is_wrong_when_spectra_differ(sylv_problem):
    """The denominators printed in eq. (5.4)/Alg. 4 (spectra swapped) disagree with eq. (5.5)."""
    *_, res = sylv_problem
    m, s = 6, res.logA.s
    lam, Q = lyap.eig_T(res.logA, m)
    ups, P = lyap.eig_T(res.logB, m)
    a = Q[:s].T @ res.logA.gamma
    b = P[:s].T @ res.logB.gamma
    F = Q[-s:].T @ res.logA.tau_next[m - 1].T
    G = P[-s:].T @ res.logB.tau_next[m - 1].T
    printed = 0.0
    for i in range(s * m):
        printed += np.sum((((a[i] @ b.T) / (ups[i] + lam)) @ G) ** 2)
        printed += np.sum((((a @ b[i]) / (lam[i] + ups)) @ F) ** 2)
    ref, _ = _reduced_bs(res, m)
    assert abs(np.sqrt(printed) - ref) > 1e-3 * ref


def test_symmetric_case_reduces_to_lyapunov():
    """B = A, C2 = C1: eq. (5.5) becomes 2||Y E_m tau^T||^2 and the histories coincide (P7)."""
    A = wl.laplacian_2d(9)
    C = wl.rhs(81, 2, 6)
    ly = lyap.solve(A, C, tol=0.0, maxit=15)
    sy = sylvester.solve(A, A, C, C, tol=0.0, maxit=15)
    assert np.allclose(sy.history, ly.history, rtol=1e-10, atol=0)


def test_factors_solve_full_equation():
    """Z1 Z2^T against Bartels-Stewart on the full (small) equation."""
    A = wl.laplacian_2d(10)
    B = wl.paper_ex64_operator_B(8)
    C1 = wl.rhs(100, 2, 1)
    C2 = wl.rhs(64, 2, 2)
    res = sylvester.solve(A, B, C1, C2, tol=1e-11, maxit=200)
    assert res.converged
    Z1, Z2, _ = sylvester.factor(A, B, C1, C2, res, trunc_eps=1e-14)
    X = sla.solve_sylvester(A.toarray(), B.toarray(), -C1 @ C2.T)
    assert np.linalg.norm(Z1 @ Z2.T - X) <= 1e-8 * np.linalg.norm(X)
    d = explicit.sylv_dense(A, B, Z1, Z2, C1, C2)
    lr = explicit.sylv_lowrank(A, B, Z1, Z2, C1, C2)
    assert abs(d - lr) <= 1e-8 * d + 1e-12
