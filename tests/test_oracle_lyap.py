"""Pins for the FP64 Lyapunov oracle against things other than itself.

Each test fixes the oracle to mathematics the paper states: the Bartels-Stewart
solution of the reduced equation (eq. 2.3) with the residual identity (eq. 2.4),
the explicit residual of the full equation, the Galerkin condition (eq. 2.1),
a closed-form solution (Kronecker/sine eigenbasis of the Laplacian), the
diagonal case, textbook scalar Lanczos (s = 1), invariants, and the planted
mistakes at the end, which must make one of those pins fail.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import workloads as wl
from oracle import explicit, lyap


def _reduced_bs_residual(log, m):
    """sqrt(2) ||Y_m E_m tau_{m+1,m}^T||_F with Y_m from Bartels-Stewart (eqs. 2.3, 2.4)."""
    s = log.s
    T = lyap.dense_T(log, m)
    E1g = np.zeros((s * m, s))
    E1g[:s, :] = log.gamma
    Y = sla.solve_continuous_lyapunov(T, -E1g @ E1g.T)
    return np.sqrt(2.0) * np.linalg.norm(Y[:, -s:] @ log.tau_next[m - 1].T, "fro"), Y, T


@pytest.fixture(scope="module")
def small_problem():
    n, s = 90, 3
    A = wl.random_snd_dense(n, seed=7, lam_min=1.0, lam_max=300.0)
    C = wl.rhs(n, s, seed=3)
    res = lyap.solve(A, C, tol=0.0, maxit=12, keep_basis=True)
    return A, C, res


def test_qr_pos_reconstructs():
    W = wl.rhs(50, 4, 11)
    V, R = lyap.qr_pos(W)
    assert np.all(np.diag(R) > 0)
    assert np.allclose(np.triu(R), R)
    assert np.linalg.norm(V @ R - W) < 1e-13 * np.linalg.norm(W)
    assert np.linalg.norm(V.T @ V - np.eye(4)) < 1e-14


def test_cheap_residual_equals_bartels_stewart(small_problem):
    """Prop. 3.1 == sqrt(2)||Y E_m tau^T|| with Y from a Schur-based solver (P3)."""
    _, _, res = small_problem
    for m in range(1, res.m + 1):
        ref, Y, T = _reduced_bs_residual(res.log, m)
        got = res.history[m - 1] * res.log.beta**2
        assert abs(got - ref) <= 1e-10 * ref, (m, got, ref)


def test_cheap_residual_equals_explicit_full_residual(small_problem):
    """eq. (2.4): ||A X_m + X_m A + C C^T||_F with X_m = V_m Y_m V_m^T, and the Galerkin condition."""
    A, C, res = small_problem
    s = res.log.s
    for m in (1, 2, 5, 9, 12):
        _, Y, _ = _reduced_bs_residual(res.log, m)
        Vm = np.hstack(res.log.basis[:m])
        X = Vm @ Y @ Vm.T
        R = A @ X + X @ A + C @ C.T
        full = np.linalg.norm(R, "fro") / res.log.beta**2
        assert abs(full - res.history[m - 1]) <= 1e-9 * res.history[m - 1], (m, full, res.history[m - 1])
        # Galerkin: V_m^T R_m V_m = 0 (eq. 2.1)
        assert np.linalg.norm(Vm.T @ R @ Vm) <= 1e-10 * np.linalg.norm(C @ C.T)
        assert Vm.shape[1] == s * m


def test_T_is_projection_of_A(small_problem):
    """T_m = V_m^T A V_m (Sec. 2) and the three-term recurrence (eq. 2.6)."""
    A, _, res = small_problem
    m = 8
    Vm = np.hstack(res.log.basis[:m])
    T = lyap.dense_T(res.log, m)
    assert np.linalg.norm(Vm.T @ A @ Vm - T) <= 1e-11 * np.linalg.norm(A, 2)
    s = res.log.s
    for j in range(1, m):
        Vj = res.log.basis[j]
        lhs = A @ Vj
        rhs = Vj @ res.log.tau_diag[j] + res.log.basis[j + 1] @ res.log.tau_next[j] + res.log.basis[j - 1] @ res.log.tau_prev[j]
        assert np.linalg.norm(lhs - rhs) <= 1e-11 * np.linalg.norm(lhs)
        # tau_{j-1,j} equals tau_{j,j-1}^T in exact arithmetic
        assert np.linalg.norm(res.log.tau_prev[j] - res.log.tau_next[j - 1].T) <= 1e-10 * np.linalg.norm(A, 2)


def test_invariants(small_problem):
    A, C, res = small_problem
    V = np.hstack(res.log.basis)
    # local orthogonality is enforced by Alg. 2; global orthogonality degrades slowly
    for j in range(len(res.log.basis) - 1):
        Vj, Vn = res.log.basis[j], res.log.basis[j + 1]
        assert np.linalg.norm(Vj.T @ Vj - np.eye(Vj.shape[1])) < 1e-14
        assert np.linalg.norm(Vn.T @ Vj) < 1e-13
    assert np.linalg.norm(V.T @ V - np.eye(V.shape[1]), 2) < 1e-10
    lam, Q = lyap.eig_T(res.log, res.m)
    assert np.all(lam < 0)
    assert np.all(lam[:, None] + lam[None, :] < 0)
    # sign flip of any eigenvector leaves the residual unchanged (P6)
    flip = np.where(np.random.default_rng(0).random(lam.shape[0]) < 0.5, -1.0, 1.0)
    r1 = lyap.cheap_residual(lam, Q, res.log.gamma, res.log.tau_next[res.m - 1], res.log.s)
    r2 = lyap.cheap_residual(lam, Q * flip, res.log.gamma, res.log.tau_next[res.m - 1], res.log.s)
    assert abs(r1 - r2) <= 1e-13 * r1
    # scale invariance of the relative residual under A -> cA, C -> cC
    res2 = lyap.solve(3.5 * A, 0.25 * C, tol=0.0, maxit=res.m)
    assert np.allclose(res2.history, res.history, rtol=1e-9, atol=0)


def test_scalar_case_is_textbook_lanczos():
    """s = 1: T_m is the tridiagonal of the textbook Lanczos recurrence (P7)."""
    A = wl.laplacian_2d(12)
    b = wl.rhs(A.shape[0], 1, 5)[:, 0]
    m = 15
    # textbook recurrence with full reorthogonalisation (a different algorithm)
    Vs = [b / np.linalg.norm(b)]
    alphas, betas = [], []
    for j in range(m):
        w = A @ Vs[j]
        alphas.append(Vs[j] @ w)
        Vmat = np.array(Vs).T
        w = w - Vmat @ (Vmat.T @ w)
        w = w - Vmat @ (Vmat.T @ w)
        betas.append(np.linalg.norm(w))
        Vs.append(w / betas[-1])
    res = lyap.solve(A, b[:, None], tol=0.0, maxit=m)
    ab = lyap.band_T(res.log, m)
    scale = np.abs(alphas).max()
    assert np.allclose(ab[0], alphas, atol=1e-10 * scale, rtol=0)
    assert np.allclose(np.abs(ab[1, : m - 1]), betas[: m - 1], atol=1e-10 * scale, rtol=0)
    assert abs(res.log.tau_next[m - 1][0, 0] - betas[m - 1]) <= 1e-10 * scale


def _sine_basis(k):
    j = np.arange(1, k + 1)
    U = np.sqrt(2.0 / (k + 1)) * np.sin(np.outer(j, j) * np.pi / (k + 1))
    h = 1.0 / (k + 1)
    mu = -(4.0 / h**2) * np.sin(j * np.pi * h / 2) ** 2
    return U, mu


def test_closed_form_laplacian_solution():
    """P1: X = -U [(U^T C C^T U)_pq / (mu_p + mu_q)] U^T in the Kronecker sine basis."""
    k, s = 12, 2
    A = wl.laplacian_2d(k)
    C = wl.rhs(k * k, s, 21)
    U1, mu1 = _sine_basis(k)
    U = np.kron(U1, U1)                   # x fastest within y: kron(U_y, U_x)
    mu = (mu1[:, None] + mu1[None, :]).ravel()
    assert np.linalg.norm(A @ U - U * mu) < 1e-9 * np.abs(mu).max()
    G = U.T @ C
    X = -U @ ((G @ G.T) / (mu[:, None] + mu[None, :])) @ U.T
    res = lyap.solve(A, C, tol=1e-11, maxit=200)
    assert res.converged
    Z, _ = lyap.factor(A, C, res, trunc_eps=1e-14)
    err = np.linalg.norm(Z @ Z.T - X) / np.linalg.norm(X)
    assert err < 1e-9, err
    lam, _ = lyap.eig_T(res.log, res.m)
    assert lam.min() >= mu.min() * (1 + 1e-12) and lam.max() <= mu.max() * (1 - 1e-12)


def test_diagonal_matrix_fills_space():
    """P7: A = diag(d); once s*m = n the residual vanishes and X_ij = -(CC^T)_ij/(d_i+d_j)."""
    n = 24
    d = -np.linspace(1.0, 40.0, n)
    A = sp.diags(d).tocsr()
    C = wl.rhs(n, 1, 2)
    res = lyap.solve(A, C, tol=0.0, maxit=n)
    assert res.history[-1] < 1e-9
    X = -(C @ C.T) / (d[:, None] + d[None, :])
    V = np.hstack(list(lyap.regenerate_basis(A, C, res.log, n)))
    Y = sla.solve_continuous_lyapunov(lyap.dense_T(res.log, n), -np.outer(np.eye(n)[:, 0], np.eye(n)[:, 0]) * res.log.gamma[0, 0] ** 2)
    assert np.linalg.norm(V @ Y @ V.T - X) < 1e-6 * np.linalg.norm(X)


def test_two_pass_matches_stored_basis(small_problem):
    """P10: the second pass regenerates the basis and Z up to rounding."""
    A, C, res = small_problem
    Zs, _ = lyap.factor(A, C, res, two_pass=False)
    Zt, _ = lyap.factor(A, C, res, two_pass=True)
    assert np.linalg.norm(Zs - Zt) <= 1e-10 * np.linalg.norm(Zs)
    for j, Vj in enumerate(lyap.regenerate_basis(A, C, res.log, res.m)):
        assert np.linalg.norm(Vj - res.log.basis[j]) < 1e-10


def test_truncation_rule():
    """eq. (2.5): ||Y~ - Ycheck Ycheck^T||_F <= eps, and dropping one more value exceeds eps."""
    A = wl.laplacian_2d(10)
    C = wl.rhs(100, 2, 4)
    res = lyap.solve(A, C, tol=1e-9, maxit=200)
    beta2 = res.log.beta**2
    for te in (1e-12, 1e-8, 1e-5):
        M, sig = lyap.truncated_factor(res.log, res.m, trunc_eps=te)
        lam, Q = lyap.eig_T(res.log, res.m)
        a = Q[:2, :].T @ res.log.gamma
        Yt = -(a @ a.T) / (lam[:, None] + lam[None, :])
        Yc = Q.T @ M
        assert np.linalg.norm(Yt - Yc @ Yc.T) <= te * beta2 * (1 + 1e-8) + 1e-14 * np.linalg.norm(Yt)
        allsig = np.sort(np.linalg.eigvalsh(Yt))[::-1]
        t = sig.shape[0]
        if t > 0:
            assert np.linalg.norm(allsig[t - 1:]) > te * beta2


def test_explicit_lowrank_equals_dense():
    n, t, s = 60, 5, 2
    A = wl.random_snd_dense(n, 3)
    Z = wl.rhs(n, t, 8)
    C = wl.rhs(n, s, 9)
    d = explicit.lyap_dense(A, Z, C)
    l = explicit.lyap_lowrank(A, Z, C)
    assert abs(d - l) <= 1e-12 * d


def test_config_c1_explicit_residual():
    """The factor returned at convergence satisfies the full equation to the tolerance
    plus the truncation's contribution 2||A||_2 eps (eq. 2.5)."""
    P = wl.config_c1(0)
    res = lyap.solve(P.A, P.C1, tol=P.tol, maxit=P.maxit)
    assert res.converged
    Z, _ = lyap.factor(P.A, P.C1, res)
    rel = explicit.lyap_lowrank(P.A, Z, P.C1) / res.log.beta**2
    normA = 8.0 * 51**2
    assert rel <= P.tol + 2 * normA * 1e-12 + 1e-10
    assert explicit.lyap_dense(P.A, Z, P.C1) == pytest.approx(rel * res.log.beta**2, rel=1e-8)


def test_paper_example_61_iteration_count():
    """Loose pin to the paper's printed iteration count (Example 6.1, s = 1)."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_ex61_iterations.json")))
    case = gold["cases"]["s1"]
    A = wl.paper_ex61_operator(gold["grid"])
    C = wl.paper_rand_rhs(A.shape[0], 1, seed=0)
    res = lyap.solve(A, C, tol=gold["tol"], maxit=2 * case["iterations"])
    assert res.converged
    assert abs(res.m - case["iterations"]) <= gold["rel_window"] * case["iterations"], res.m


# ----------------------------------------------------------------------------
# Planted mistakes: each variant of the oracle must fail at least one pin.
# ----------------------------------------------------------------------------

def _bs_mismatch(res, cheap_fn):
    worst = 0.0
    for m in range(1, res.m + 1):
        ref, _, _ = _reduced_bs_residual(res.log, m)
        lam, Q = lyap.eig_T(res.log, m)
        got = cheap_fn(lam, Q, res.log.gamma, res.log.tau_next[m - 1], res.log.s)
        worst = max(worst, abs(got - ref) / ref)
    return worst


def _mut_no_sqrt2(lam, Q, g, tau, s):
    return lyap.cheap_residual(lam, Q, g, tau, s) / np.sqrt(2.0)


def _mut_tau_transposed(lam, Q, g, tau, s):
    return lyap.cheap_residual(lam, Q, g, tau.T, s)


def _mut_first_rows_for_W(lam, Q, g, tau, s):
    a = Q[:s, :].T @ g
    Wm = Q[:s, :].T @ tau.T
    r = sum(float(np.sum(((a[i] @ a.T) / (lam[i] + lam) @ Wm) ** 2)) for i in range(lam.shape[0]))
    return np.sqrt(2 * r)


def _mut_gamma_transposed(lam, Q, g, tau, s):
    return lyap.cheap_residual(lam, Q, g.T, tau, s)


def _mut_denominator_minus(lam, Q, g, tau, s):
    a = Q[:s, :].T @ g
    Wm = Q[-s:, :].T @ tau.T
    r = 0.0
    for i in range(lam.shape[0]):
        den = lam[i] - lam
        den[i] = 2 * lam[i]
        r += float(np.sum(((a[i] @ a.T) / den @ Wm) ** 2))
    return np.sqrt(2 * r)


@pytest.mark.parametrize("mut", [_mut_no_sqrt2, _mut_tau_transposed, _mut_first_rows_for_W,
                                 _mut_gamma_transposed, _mut_denominator_minus])
def test_planted_mistakes_are_caught(small_problem, mut):
    _, _, res = small_problem
    assert _bs_mismatch(res, lyap.cheap_residual) < 1e-10
    assert _bs_mismatch(res, mut) > 1e-6


def test_planted_mistake_in_recurrence_is_caught(small_problem, monkeypatch):
    """Dropping the second MGS sweep or the tau_{j-1,j} term breaks the projection pin."""
    A, C, _ = small_problem
    orig = lyap.lanczos_step

    def one_sweep(A_, Vp, Vc):
        s = Vc.shape[1]
        W = A_ @ Vc
        tp = np.zeros((s, s))
        if Vp is not None:
            tp = Vp.T @ W
        td = Vc.T @ W
        W = W - Vc @ td      # forgets W -= Vp tp
        Vn, tn = lyap.qr_pos(W)
        return Vn, tp, td, tn

    monkeypatch.setattr(lyap, "lanczos_step", one_sweep)
    bad = lyap.solve(A, C, tol=0.0, maxit=8, keep_basis=True)
    monkeypatch.setattr(lyap, "lanczos_step", orig)
    Vm = np.hstack(bad.log.basis[:8])
    assert np.linalg.norm(Vm.T @ A @ Vm - lyap.dense_T(bad.log, 8)) > 1e-6 * np.linalg.norm(A, 2)


def test_truncation_threshold_tied_to_tol():
    """Reading of eq. 2.5 (eps tied to the residual target): with eps = 1e-12 (the paper's value
    at ||C|| = 1, tol 1e-6) the truncation alone leaves an explicit residual far above a tol of
    1e-10 on these Laplacians (||A|| ~ 1e4); with eps = min(1e-12, tol / (20 ||T_m||)) the
    explicit residual of the factor equals the cheap residual to 1%, which the residual bound
    2 ||A|| eps <= tol / 10 predicts."""
    for k, s in ((40, 2), (30, 1), (24, 3)):
        A = wl.laplacian_2d(k)
        C = wl.rhs(A.shape[0], s, 3)
        res = lyap.solve(A, C, tol=1e-10, maxit=400)
        b2 = np.linalg.norm(C) ** 2
        Z12, _ = lyap.factor(A, C, res, trunc_eps=1e-12)
        Za, _ = lyap.factor(A, C, res)
        r12 = explicit.lyap_lowrank(A, Z12, C) / b2
        ra = explicit.lyap_lowrank(A, Za, C) / b2
        assert r12 > 10 * res.history[-1]
        assert abs(ra - res.history[-1]) <= 1e-2 * res.history[-1]
        assert Za.shape[1] > Z12.shape[1]
        lam, _ = lyap.eig_T(res.log, res.m)
        assert lyap.auto_trunc_eps(1e-10, np.max(np.abs(lam))) == 1e-10 / (20 * np.max(np.abs(lam)))
    assert lyap.auto_trunc_eps(1e-6, 1.0) == 1e-12  # the paper's eps where it is already small enough
