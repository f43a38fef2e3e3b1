"""FP64 oracle for A X + X B + C1 C2^T = 0 with A large and B small (Sec. 5.2, Alg. 5).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Only A is projected.  X_m = V_m Y_m, with V_m the block Lanczos basis of K_m(A, C1) and
C1 = V_1 gamma_1; the Galerkin condition V_m^T R_m = 0 gives the reduced equation

    T_m Y_m + Y_m B + E_1 gamma_1 C2^T = 0        (sm x n2).

B = P Upsilon P^T is diagonalised once.  With T_m = Q Lambda Q^T,
Y_m = Q Y~ P^T and Y~_ij = -(Q^T E_1 gamma_1 C2^T P)_ij / (lambda_i + upsilon_j).

Since A V_m = V_m T_m + V_{m+1} tau_{m+1,m} E_m^T, the residual is
R_m = V_{m+1} tau_{m+1,m} E_m^T Y_m, so ||R_m||_F = ||tau_{m+1,m} E_m^T Y_m||_F.  Alg. 5
evaluates it without Y_m: S = (P^T C2 gamma_1^T)(E_1^T Q) (n2 x sm),
W = (Q^T E_m) tau_{m+1,m}^T, and ||R_m||_F^2 = sum_j ||(e_j^T S) D_j^{-1} W||^2 with
D_j = upsilon_j I + Lambda.  The relative residual divides by ||C1||_F ||C2||_F, as in the
two-sided case.  The factors are Z1 = V_m (Q Y1) and Z2 = P Y2 from the truncated SVD
Y~ ~= Y1 Y2^T (the end of Sec. 5.2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lyap


def eig_B(B):
    """B = P Upsilon P^T (dense symmetric eigendecomposition, once per solve)."""
    Bd = B.toarray() if hasattr(B, "toarray") else np.asarray(B, dtype=np.float64)
    ups, P = np.linalg.eigh(0.5 * (Bd + Bd.T))
    return ups, P


def cheap_residual(lam, Q, ups, P, gamma, C2, tau, s):
    """||R_m||_F by Alg. 5."""
    S = (P.T @ C2 @ gamma.T) @ Q[:s, :]     # (P^T C2 gamma_1^T)(E_1^T Q)
    W = Q[-s:, :].T @ tau.T                  # (Q^T E_m) tau^T
    res = 0.0
    for j in range(ups.shape[0]):
        v = (S[j] / (ups[j] + lam)) @ W      # (e_j^T S) D_j^{-1} W
        res += float(v @ v)
    return np.sqrt(res)


def reduced_solution(log: lyap.LanczosLog, m: int, ups, P, C2):
    """Y~ (sm x n2) and the eigenpairs of T_m."""
    s = log.s
    lam, Q = lyap.eig_T(log, m)
    G = (Q[:s, :].T @ log.gamma) @ (C2.T @ P)   # Q^T E_1 gamma_1 C2^T P
    return -G / (lam[:, None] + ups[None, :]), lam, Q


@dataclass
class SmallBResult:
    log: lyap.LanczosLog
    ups: np.ndarray
    P: np.ndarray
    history: np.ndarray
    m: int
    converged: bool


def residual_at(log: lyap.LanczosLog, m: int, ups, P, C2) -> float:
    lam, Q = lyap.eig_T(log, m)
    res = cheap_residual(lam, Q, ups, P, log.gamma, C2, log.tau_next[m - 1], log.s)
    return res / (log.beta * float(np.linalg.norm(C2, "fro")))


def solve(A, B, C1, C2, tol=1e-8, maxit=1000, keep_basis=False) -> SmallBResult:
    """Block Lanczos on (A, C1) (Alg. 2) with the check of Alg. 5 after every step."""
    C2 = np.asarray(C2, dtype=np.float64)
    ups, P = eig_B(B)
    V1, log = lyap.start(C1, keep_basis)
    Vprev, Vcur = None, V1
    hist, converged, m = [], False, 0
    for j in range(1, maxit + 1):
        Vnext, tp, td, tn = lyap.lanczos_step(A, Vprev, Vcur)
        log.tau_prev.append(tp)
        log.tau_diag.append(td)
        log.tau_next.append(tn)
        if log.basis is not None:
            log.basis.append(Vnext)
        Vprev, Vcur = Vcur, Vnext
        m = j
        rel = residual_at(log, j, ups, P, C2)
        hist.append(rel)
        if rel <= tol:
            converged = True
            break
    return SmallBResult(log, ups, P, np.array(hist), m, converged)


def factor(A, C1, C2, res: SmallBResult, trunc_eps=1e-12):
    """Z1 = V_m (Q Y1) by the two-pass device and Z2 = P Y2, with Y~ ~= Y1 Y2^T truncated so
    that the discarded singular values have Frobenius norm <= trunc_eps ||C1||_F ||C2||_F."""
    log, m, s = res.log, res.m, res.log.s
    C2 = np.asarray(C2, dtype=np.float64)
    Yt, lam, Q = reduced_solution(log, m, res.ups, res.P, C2)
    U, sig, Vt = np.linalg.svd(Yt, full_matrices=False)
    eps_abs = trunc_eps * log.beta * float(np.linalg.norm(C2, "fro"))
    tail = np.sqrt(np.concatenate([np.cumsum((sig**2)[::-1])[::-1], [0.0]]))
    t = int(np.argmax(tail <= eps_abs))
    r = np.sqrt(sig[:t])
    M1 = Q @ (U[:, :t] * r)
    Z2 = res.P @ (Vt[:t, :].T * r)
    Z1 = np.zeros((C1.shape[0], t))
    for j, Vj in enumerate(lyap.regenerate_basis(A, C1, log, m)):
        Z1 += Vj @ M1[j * s:(j + 1) * s, :]
    return Z1, Z2, sig[:t]
