"""FP64 oracle for the generalised Lyapunov equation A X E + E X A + C C^T = 0 with E
symmetric positive definite (the example with a mass matrix in Sec. 6).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 6 treats this equation as a standard Lyapunov equation when E is symmetric positive
definite.  The reading taken here: with the Cholesky factor E = L L^T, X~ = L^T X L solves

    A~ X~ + X~ A~ + C~ C~^T = 0,   A~ = L^{-1} A L^{-T},   C~ = L^{-1} C,

since L^{-1}(A X E + E X A)L^{-T} = A~ X~ + X~ A~.  A~ is symmetric negative definite, so
Alg. 1-3 run on it unchanged, and a factor X~ ~= Z~ Z~^T gives X ~= Z Z^T with
Z = L^{-T} Z~.  The residual the method monitors is that of the transformed equation; the
original one is R = L R~ L^T.  Dense Cholesky and triangular solves: small n only.

The factor uses the stored basis.  The two-pass device (Sec. 3.3) of ``lyap.factor`` replays
the recurrence from the logged coefficients with a rounding different from the first pass's
MGS sweeps, and on the transformed mass-matrix operators (||A~|| / |lambda_max(A~)| ~ 270)
that replay drifts from the stored basis exponentially, by about 10^3 every five steps.

For the same reason the basis loses orthogonality within a few tens of steps, after which the
residual histories of two correct implementations part company (their roundings differ).  The
default step therefore takes Alg. 2's block Gram-Schmidt (twice) against every stored block,
not only V_{j-1} and V_j: in exact arithmetic the coefficients are the same (the other
projections vanish), and in floating point the basis stays orthonormal to rounding, so the
history is a function of the operator alone.  ``reorth=False`` gives the plain step of Alg. 2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import lyap


@dataclass
class GeneralResult:
    inner: lyap.SolveResult
    L: np.ndarray       # E = L L^T
    At: np.ndarray      # A~
    Ct: np.ndarray      # C~


def transform(A, E, C):
    """A~ = L^{-1} A L^{-T} and C~ = L^{-1} C with E = L L^T."""
    Ed = E.toarray() if hasattr(E, "toarray") else np.asarray(E, dtype=np.float64)
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A, dtype=np.float64)
    L = np.linalg.cholesky(0.5 * (Ed + Ed.T))
    T1 = sla.solve_triangular(L, Ad, lower=True)          # L^{-1} A
    At = sla.solve_triangular(L, T1.T, lower=True).T      # (L^{-1} A) L^{-T}
    At = 0.5 * (At + At.T)
    Ct = sla.solve_triangular(L, np.asarray(C, dtype=np.float64), lower=True)
    return L, At, Ct


def lanczos_step_full(A, basis, Vcur):
    """Alg. 2's step with the block Gram-Schmidt run (twice) against every stored block: W = A V_j;
    for l = 1, 2 and i = 1..j: alpha = V_i^T W, W -= V_i alpha, with tau_{j-1,j} and tau_jj the sums
    of the alphas of V_{j-1} and V_j; finally W = V_{j+1} tau_{j+1,j}.  ``basis`` holds V_1..V_j."""
    s = Vcur.shape[1]
    W = A @ Vcur
    tau_prev = np.zeros((s, s))
    tau_diag = np.zeros((s, s))
    j = len(basis)
    for _ in range(2):
        for i, Vi in enumerate(basis, start=1):
            alpha = Vi.T @ W
            if i == j:
                tau_diag += alpha
            elif i == j - 1:
                tau_prev += alpha
            W = W - Vi @ alpha
    Vnext, tau_next = lyap.qr_pos(W)
    return Vnext, tau_prev, tau_diag, tau_next


def solve_full(A, C, tol=1e-8, maxit=1000) -> lyap.SolveResult:
    """Algorithm 1 (steps 1-7) with ``lanczos_step_full``; the check is Prop. 3.1 at every m."""
    V1, log = lyap.start(C, keep_basis=True)
    hist, converged, m = [], False, 0
    for j in range(1, maxit + 1):
        Vnext, tp, td, tn = lanczos_step_full(A, log.basis[:j], log.basis[j - 1])
        log.tau_prev.append(tp)
        log.tau_diag.append(td)
        log.tau_next.append(tn)
        log.basis.append(Vnext)
        m = j
        rel = lyap.residual_at(log, j)
        hist.append(rel)
        if rel <= tol:
            converged = True
            break
    return lyap.SolveResult(log=log, history=np.array(hist), m=m, converged=converged, tol=tol)


def solve(A, E, C, tol=1e-8, maxit=1000, reorth=True) -> GeneralResult:
    L, At, Ct = transform(A, E, C)
    inner = solve_full(At, Ct, tol=tol, maxit=maxit) if reorth else lyap.solve(At, Ct, tol=tol, maxit=maxit,
                                                                                keep_basis=True)
    return GeneralResult(inner, L, At, Ct)


def factor(res: GeneralResult, trunc_eps: float = 1e-12):
    """Z with X ~= Z Z^T: the factor of the transformed equation from the stored basis, mapped
    by L^{-T}."""
    Zt, sig = lyap.factor(res.At, res.Ct, res.inner, trunc_eps=trunc_eps, two_pass=False)
    return sla.solve_triangular(res.L.T, Zt, lower=False), sig
