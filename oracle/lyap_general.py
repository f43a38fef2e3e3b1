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


def solve(A, E, C, tol=1e-8, maxit=1000) -> GeneralResult:
    L, At, Ct = transform(A, E, C)
    return GeneralResult(lyap.solve(At, Ct, tol=tol, maxit=maxit, keep_basis=True), L, At, Ct)


def factor(res: GeneralResult, trunc_eps: float = 1e-12):
    """Z with X ~= Z Z^T: the factor of the transformed equation from the stored basis, mapped
    by L^{-T}."""
    Zt, sig = lyap.factor(res.At, res.Ct, res.inner, trunc_eps=trunc_eps, two_pass=False)
    return sla.solve_triangular(res.L.T, Zt, lower=False), sig
