"""FP64 oracle for the extended Krylov space K_m(A, C) + K_m(A^{-1}, A^{-1} C) (Sec. 4).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The inner solves with A are exact here
(a sparse LU of A); the CUDA path replaces them by preconditioned conjugate gradients.

Basis blocks V_j = [V_j^(1), V_j^(2)] have 2s columns.  The start is the QR factorisation
[C, A^{-1} C] = V_1 gamma (Sec. 4), so C = V_1 gamma(:, 1:s).  Step j forms
W = [A V_j^(1), A^{-1} V_j^(2)], orthogonalises it by block MGS (twice) and takes its QR.

Readings of the paper taken here:
  * Sec. 4 states that Alg. 2 (orthogonalisation against V_{j-1} and V_j only) can build this
    basis, the coefficients against older blocks vanishing in exact arithmetic.  In floating
    point that short recurrence loses orthogonality by a factor of about 30 per step on a
    Laplacian (the solve with A amplifies the rounding left in older directions; the pins show
    it), so W is orthogonalised against every previous block.  This spans the same space and
    gives the same block tridiagonal T_m; the pins check that the older coefficients are at
    rounding level in the first steps.
  * T_m = V_m^T A V_m is formed by explicit projection, tau_jj = V_j^T A V_j and
    tau_{j+1,j} = V_{j+1}^T A V_j.  The paper leaves the recurrence for T_m to the extended
    Krylov literature, and inexact inner solves would break such a recurrence anyway.
  * Since A maps the extended space of dimension 2sm into that of dimension 2s(m+1),
    A V_m = V_m T_m + V_{m+1} tau_{m+1,m} E_m^T holds, so Prop. 3.1 and Alg. 3 apply unchanged
    to T_m with block size 2s, right-hand side E_1 gamma_1 gamma_1^T E_1^T (gamma_1 =
    gamma(:, 1:s)) and tau_{m+1,m} (Sec. 4); beta = ||C||_F as in the standard case.
  * The factor is formed from the stored basis (the paper's two-pass variant for the extended
    space is not part of this oracle).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import lyap


@dataclass
class EKLog:
    s: int                                            # block size of C (blocks have 2s columns)
    beta: float
    gamma: np.ndarray                                 # [C, A^{-1} C] = V_1 gamma (2s x 2s)
    basis: list = field(default_factory=list)         # V_1, V_2, ...
    tau_diag: list = field(default_factory=list)      # V_j^T A V_j
    tau_next: list = field(default_factory=list)      # V_{j+1}^T A V_j

    @property
    def gamma1(self) -> np.ndarray:
        """C = V_1 gamma_1, padded with zero columns to 2s x 2s for the check formulas."""
        g = np.zeros_like(self.gamma)
        g[:, : self.s] = self.gamma[:, : self.s]
        return g


def factor_A(A):
    """Exact inner solver: a sparse LU of A (the CUDA path uses preconditioned CG)."""
    lu = spla.splu(A.tocsc())
    return lambda B: lu.solve(np.asarray(B, dtype=np.float64))


def start(A, C, solve):
    """beta = ||C||_F and [C, A^{-1} C] = V_1 gamma."""
    C = np.asarray(C, dtype=np.float64)
    beta = float(np.linalg.norm(C, "fro"))
    V1, gamma = lyap.qr_pos(np.hstack([C, solve(C)]))
    return EKLog(s=C.shape[1], beta=beta, gamma=gamma, basis=[V1])


def step(A, solve, basis, coefs=None):
    """W = [A V_j^(1), A^{-1} V_j^(2)] for the last block of ``basis``; block MGS (twice) against
    every block of ``basis``, then QR.  ``coefs`` (a list) receives ||V_i^T W|| of the first
    sweep per block, oldest first."""
    Vcur = basis[-1]
    s = Vcur.shape[1] // 2
    W = np.hstack([A @ Vcur[:, :s], solve(Vcur[:, s:])])
    for sweep in range(2):
        for Vi in basis:
            alpha = Vi.T @ W
            if sweep == 0 and coefs is not None:
                coefs.append(float(np.linalg.norm(alpha)))
            W = W - Vi @ alpha
    Vnext, _ = lyap.qr_pos(W)
    return Vnext


def band_T(log: EKLog, m: int) -> np.ndarray:
    """Lower band (half-bandwidth 2s) of T_m from the projected blocks, symmetric part on the diagonal."""
    S = 2 * log.s
    N = S * m
    T = np.zeros((N, N))
    for j in range(m):
        D = log.tau_diag[j]
        T[j * S:(j + 1) * S, j * S:(j + 1) * S] = 0.5 * (D + D.T)
        if j + 1 < m:
            T[(j + 1) * S:(j + 2) * S, j * S:(j + 1) * S] = log.tau_next[j]
            T[j * S:(j + 1) * S, (j + 1) * S:(j + 2) * S] = log.tau_next[j].T
    ab = np.zeros((S + 1, N))
    for d in range(S + 1):
        ab[d, : N - d] = np.diagonal(T, -d)
    return ab


def residual_at(log: EKLog, m: int) -> float:
    """||R_m||_F / beta^2 by Prop. 3.1 on the extended T_m (block size 2s)."""
    S = 2 * log.s
    lam, Q = sla.eig_banded(band_T(log, m), lower=True)
    res = lyap.cheap_residual(lam, Q, log.gamma1, log.tau_next[m - 1], S)
    return res / log.beta**2


@dataclass
class EKResult:
    log: EKLog
    history: np.ndarray
    m: int
    converged: bool
    tol: float = 1e-8


def solve(A, C, tol=1e-8, maxit=200, inner=None) -> EKResult:
    """Galerkin projection onto the extended Krylov space (Alg. 1 with Sec. 4's space)."""
    inv = inner if inner is not None else factor_A(A)
    log = start(A, C, inv)
    hist, converged, m = [], False, 0
    for j in range(1, maxit + 1):
        Vcur = log.basis[-1]
        Vnext = step(A, inv, log.basis)
        AV = A @ Vcur
        log.tau_diag.append(Vcur.T @ AV)
        log.tau_next.append(Vnext.T @ AV)
        log.basis.append(Vnext)
        m = j
        rel = residual_at(log, j)
        hist.append(rel)
        if rel <= tol:
            converged = True
            break
    return EKResult(log, np.array(hist), m, converged, tol)


def factor(res: EKResult, trunc_eps: float | None = None):
    """Z = V_m (Q Ycheck) with the truncation of eq. 2.5 (eps = trunc_eps beta^2; None: the
    tolerance-consistent lyap.auto_trunc_eps), stored basis."""
    log, m = res.log, res.m
    S = 2 * log.s
    lam, Q = sla.eig_banded(band_T(log, m), lower=True)
    if trunc_eps is None:
        trunc_eps = lyap.auto_trunc_eps(res.tol, float(np.max(np.abs(lam))))
    a = Q[:S, :].T @ log.gamma1
    Yt = -(a @ a.T) / (lam[:, None] + lam[None, :])
    sig, Wv = np.linalg.eigh(Yt)
    order = np.argsort(sig)[::-1]
    sig, Wv = sig[order], Wv[:, order]
    eps_abs = trunc_eps * log.beta**2
    pos = np.maximum(sig, 0.0)
    tail = np.sqrt(np.concatenate([np.cumsum((pos**2)[::-1])[::-1], [0.0]]))
    t = int(np.argmax(tail <= eps_abs))
    t = min(t, int(np.sum(sig > 0)))
    M = Q @ (Wv[:, :t] * np.sqrt(sig[:t]))
    V = np.hstack(log.basis[:m])
    return V @ M, sig[:t]
