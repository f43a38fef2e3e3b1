"""FP64 oracle for the Sylvester equation A X + X B + C1 C2^T = 0, A and B large (Sec. 5.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Two block Lanczos
recurrences, (A, C1) giving V_m, T_m, tau and (B, C2) giving U_m, J_m, iota,
advance together; the check at m uses both band eigendecompositions.

Reading of the paper taken here: eq. (5.4) and Algorithm 4 print the
denominator with the two spectra swapped.  The diagonalised reduced equation
Lambda Y~ + Y~ Upsilon + S = 0 gives Y~_ij = -S_ij / (lambda_i + upsilon_j), so
row i of S pairs with (lambda_i I + Upsilon)^{-1} G and column j with
(upsilon_j I + Lambda)^{-1} F.  The tests pin this against scipy's
Bartels-Stewart solve of the reduced problem and against eq. (5.5).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lyap


@dataclass
class SylvResult:
    logA: lyap.LanczosLog
    logB: lyap.LanczosLog
    history: np.ndarray
    m: int
    converged: bool
    tol: float = 1e-8


def cheap_residual(lam, Q, ups, P, g1, g2, tau, iota, s):
    """||R_m||_F without Y_m (Algorithm 4 with the corrected pairing).

    S = (Q^T E_1 g1)(g2^T E_1^T P), F = Q^T E_m tau^T, G = P^T E_m iota^T;
    ||R||^2 = sum_i ||e_i^T S (lambda_i I + Upsilon)^{-1} G||^2
            + sum_j ||(S e_j)^T (upsilon_j I + Lambda)^{-1} F||^2.
    """
    a = Q[:s, :].T @ g1
    b = P[:s, :].T @ g2
    F = Q[-s:, :].T @ tau.T
    G = P[-s:, :].T @ iota.T
    res = 0.0
    for i in range(lam.shape[0]):
        row = (a[i] @ b.T) / (lam[i] + ups)          # e_i^T S (lambda_i + Upsilon)^{-1}
        v = row @ G
        res += float(v @ v)
    for j in range(ups.shape[0]):
        col = (a @ b[j]) / (lam + ups[j])            # (S e_j)^T (upsilon_j + Lambda)^{-1}
        v = col @ F
        res += float(v @ v)
    return np.sqrt(res)


def residual_at(logA, logB, m):
    lam, Q = lyap.eig_T(logA, m)
    ups, P = lyap.eig_T(logB, m)
    res = cheap_residual(lam, Q, ups, P, logA.gamma, logB.gamma,
                         logA.tau_next[m - 1], logB.tau_next[m - 1], logA.s)
    return res / (logA.beta * logB.beta)


def solve(A, B, C1, C2, tol=1e-8, maxit=1000, check_every=1, keep_basis=False) -> SylvResult:
    """Galerkin projection with K_m(A, C1) and K_m(B, C2) of equal dimension s*m."""
    V1, logA = lyap.start(C1, keep_basis)
    U1, logB = lyap.start(C2, keep_basis)
    state = {"A": (None, V1), "B": (None, U1)}
    hist, converged, m = [], False, 0
    for j in range(1, maxit + 1):
        for key, op, log in (("A", A, logA), ("B", B, logB)):
            Vp, Vc = state[key]
            Vn, tp, td, tn = lyap.lanczos_step(op, Vp, Vc)
            log.tau_prev.append(tp)
            log.tau_diag.append(td)
            log.tau_next.append(tn)
            if log.basis is not None:
                log.basis.append(Vn)
            state[key] = (Vc, Vn)
        m = j
        if j % check_every == 0:
            rel = residual_at(logA, logB, j)
            hist.append(rel)
            if rel <= tol:
                converged = True
                break
        else:
            hist.append(np.nan)
    return SylvResult(logA, logB, np.array(hist), m, converged, tol)


def truncated_factors(logA, logB, m, trunc_eps=None, tol=None):
    """Truncated SVD of Y~ (Sec. 5.1): Y~ ~= Y1 Y2^T with ||tail||_F <= eps.

    Returns M1 = Q Y1 and M2 = P Y2 (each s*m x t) and the kept singular values;
    eps = trunc_eps * ||C1||_F ||C2||_F (trunc_eps None: lyap.auto_trunc_eps(tol, ||T_m||, ||J_m||)).
    """
    s = logA.s
    lam, Q = lyap.eig_T(logA, m)
    ups, P = lyap.eig_T(logB, m)
    if trunc_eps is None:
        trunc_eps = lyap.auto_trunc_eps(tol, float(np.max(np.abs(lam))), float(np.max(np.abs(ups))))
    a = Q[:s, :].T @ logA.gamma
    b = P[:s, :].T @ logB.gamma
    Yt = -(a @ b.T) / (lam[:, None] + ups[None, :])
    U, sig, Vt = np.linalg.svd(Yt)
    eps_abs = trunc_eps * logA.beta * logB.beta
    tail = np.sqrt(np.concatenate([np.cumsum((sig**2)[::-1])[::-1], [0.0]]))
    t = int(np.argmax(tail <= eps_abs))
    r = np.sqrt(sig[:t])
    return Q @ (U[:, :t] * r), P @ (Vt[:t, :].T * r), sig[:t]


def factor(A, B, C1, C2, res: SylvResult, trunc_eps=None):
    """Z1 = V_m (Q Y1), Z2 = U_m (P Y2), both by the two-pass device (6s stored vectors)."""
    s, m = res.logA.s, res.m
    M1, M2, sig = truncated_factors(res.logA, res.logB, m, trunc_eps, res.tol)
    Z1 = np.zeros((C1.shape[0], M1.shape[1]))
    Z2 = np.zeros((C2.shape[0], M2.shape[1]))
    for j, Vj in enumerate(lyap.regenerate_basis(A, C1, res.logA, m)):
        Z1 += Vj @ M1[j * s:(j + 1) * s, :]
    for j, Uj in enumerate(lyap.regenerate_basis(B, C2, res.logB, m)):
        Z2 += Uj @ M2[j * s:(j + 1) * s, :]
    return Z1, Z2, sig
