"""Pins of the large-A / small-B oracle (oracle/sylvester_small.py, Sec. 5.2, Alg. 5).

  * Alg. 5's residual equals ||tau E_m^T Y_m||_F with Y_m from scipy's Bartels-Stewart solve
    of the reduced equation T_m Y + Y B = -E_1 gamma_1 C2^T.
  * It equals the explicit residual ||A X_m + X_m B + C1 C2^T||_F of X_m = V_m Y_m.
  * At convergence X_m agrees with a dense solve of the full equation, and the factors
    Z1 Z2^T reproduce X_m.
  * With n2 = 1 the equation is the shifted block system (A + b I) x = -C1 c2^T.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import lyap, sylvester_small as ss


def _problem(k=20, n2=24, s=2, seed=0):
    A = wl.laplacian_2d(k, shift=1.0)
    B = wl.random_snd_dense(n2, seed=seed + 3, lam_min=0.5, lam_max=40.0)
    C1 = wl.rhs(k * k, s, seed=seed + 1)
    C2 = wl.rhs(n2, s, seed=seed + 2)
    return A, B, C1, C2


def _reduced_rhs(log, m, C2):
    s = log.s
    E1g = np.zeros((s * m, s))
    E1g[:s, :] = log.gamma
    return E1g @ C2.T


@pytest.mark.parametrize("m", [3, 8, 15])
def test_alg5_equals_bartels_stewart_on_the_reduced_equation(m):
    A, B, C1, C2 = _problem()
    res = ss.solve(A, B, C1, C2, tol=0.0, maxit=m)
    log = res.log
    T = lyap.dense_T(log, m)
    Y = sla.solve_sylvester(T, np.asarray(B), -_reduced_rhs(log, m, C2))
    s = log.s
    direct = np.linalg.norm(log.tau_next[m - 1] @ Y[-s:, :], "fro")
    lam, Q = lyap.eig_T(log, m)
    cheap = ss.cheap_residual(lam, Q, res.ups, res.P, log.gamma, C2, log.tau_next[m - 1], s)
    assert abs(cheap - direct) <= 1e-10 * direct
    # and the reduced solution of eq. 5.7 is Q Y~ P^T
    Yt, _, Q2 = ss.reduced_solution(log, m, res.ups, res.P, C2)
    assert np.allclose(Q2 @ Yt @ res.P.T, Y, rtol=0, atol=1e-10 * np.abs(Y).max())


@pytest.mark.parametrize("m", [4, 12])
def test_alg5_equals_explicit_residual(m):
    A, B, C1, C2 = _problem()
    res = ss.solve(A, B, C1, C2, tol=0.0, maxit=m, keep_basis=True)
    log = res.log
    Vm = np.hstack(log.basis[:m])
    Yt, _, Q = ss.reduced_solution(log, m, res.ups, res.P, C2)
    X = Vm @ (Q @ Yt @ res.P.T)
    Bd = np.asarray(B)
    R = A @ X + X @ Bd + C1 @ C2.T
    explicit = np.linalg.norm(R, "fro") / (np.linalg.norm(C1) * np.linalg.norm(C2))
    assert abs(res.history[m - 1] - explicit) <= 1e-9 * explicit


def test_converged_solution_and_factors():
    A, B, C1, C2 = _problem()
    res = ss.solve(A, B, C1, C2, tol=1e-10, maxit=200)
    assert res.converged
    Bd = np.asarray(B)
    X_ref = sla.solve_sylvester(A.toarray(), Bd, -C1 @ C2.T)
    Z1, Z2, sig = ss.factor(A, C1, C2, res, trunc_eps=1e-13)
    X = Z1 @ Z2.T
    assert np.linalg.norm(X - X_ref) <= 1e-8 * np.linalg.norm(X_ref)
    R = A @ X + X @ Bd + C1 @ C2.T
    rel = np.linalg.norm(R) / (np.linalg.norm(C1) * np.linalg.norm(C2))
    assert rel <= 2e-10
    assert np.all(np.diff(sig) <= 0) and Z1.shape[1] == Z2.shape[1] <= min(Z1.shape[0], Z2.shape[0])


def test_scalar_B_is_a_shifted_block_system():
    k, s, b = 16, 2, 3.5
    A = wl.laplacian_2d(k)
    C1 = wl.rhs(k * k, s, seed=5)
    c2 = wl.rhs(1, s, seed=6)
    res = ss.solve(A, np.array([[-b]]), C1, c2, tol=1e-11, maxit=300)
    assert res.converged
    Z1, Z2, _ = ss.factor(A, C1, c2, res, trunc_eps=1e-14)
    x = Z1 @ Z2.T
    x_ref = np.linalg.solve(A.toarray() - b * np.eye(k * k), -C1 @ c2.T)
    assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
