"""FP64 oracle: Galerkin projection onto the block Krylov space for A X + X A + C C^T = 0.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function restates
one step of the paper, in its order and notation, with the canonical block
indexing used throughout this repository:

    A V_j = V_{j-1} tau_{j-1,j} + V_j tau_{jj} + V_{j+1} tau_{j+1,j},   j = 1, 2, ...

(the paper's eq. (2.6) and Algorithm 2 index the new block one lower; the
coefficient at the check of a space of dimension s*m is tau_{m+1,m} in both).

Parity status: every function here is pinned by tests/test_oracle_*.py against
closed forms, Bartels-Stewart solves, explicit residuals and invariants.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


class Breakdown(RuntimeError):
    """Rank deficiency of a new block (the paper assumes full rank, Sec. 2)."""


def qr_pos(W: np.ndarray):
    """Economy Householder QR W = V R with diag(R) > 0 (Alg. 1 step 2; Alg. 2 step 9)."""
    V, R = np.linalg.qr(W, mode="reduced")
    d = np.sign(np.diag(R))
    if np.any(d == 0):
        raise Breakdown("zero diagonal in QR: rank-deficient block")
    return V * d, d[:, None] * R


@dataclass
class LanczosLog:
    """Raw coefficients of every step, kept for the second pass (Sec. 3.3)."""

    s: int
    beta: float
    gamma: np.ndarray                                  # C = V_1 gamma
    tau_prev: list = field(default_factory=list)       # tau_{j-1,j} (zero for j = 1)
    tau_diag: list = field(default_factory=list)       # tau_{jj} as computed (not symmetrised)
    tau_next: list = field(default_factory=list)       # tau_{j+1,j} (upper triangular)
    basis: list | None = None                          # V_1..V_{m+1} when kept (debug)

    @property
    def m(self) -> int:
        return len(self.tau_diag)


def start(C: np.ndarray, keep_basis: bool = False):
    """Alg. 1 steps 1-2: beta = ||C||_F and C = V_1 gamma."""
    C = np.asarray(C, dtype=np.float64)
    beta = float(np.linalg.norm(C, "fro"))
    V1, gamma = qr_pos(C)
    log = LanczosLog(s=C.shape[1], beta=beta, gamma=gamma, basis=[V1] if keep_basis else None)
    return V1, log


def lanczos_step(A, Vprev, Vcur):
    """Alg. 2: one block Lanczos step with block MGS done twice, then QR.

    W = A V_j; for l = 1, 2 and i in (j-1, j): alpha = V_i^T W,
    tau_{i,j} += alpha, W -= V_i alpha; finally W = V_{j+1} tau_{j+1,j}.
    ``Vprev`` is None at j = 1.
    """
    s = Vcur.shape[1]
    W = A @ Vcur
    tau_prev = np.zeros((s, s))
    tau_diag = np.zeros((s, s))
    for _ in range(2):
        for which, Vi in (("prev", Vprev), ("diag", Vcur)):
            if Vi is None:
                continue
            alpha = Vi.T @ W
            if which == "prev":
                tau_prev += alpha
            else:
                tau_diag += alpha
            W = W - Vi @ alpha
    Vnext, tau_next = qr_pos(W)
    return Vnext, tau_prev, tau_diag, tau_next


def band_T(log: LanczosLog, m: int) -> np.ndarray:
    """Lower band storage of the symmetric block tridiagonal T_m (Sec. 2).

    Diagonal blocks are the symmetric part of tau_jj; the sub-diagonal blocks
    are tau_{j+1,j} (j < m), the super-diagonal blocks their transposes.
    Returns ``ab`` with ab[d, i] = T_m[i + d, i], d = 0..s.
    """
    s = log.s
    N = s * m
    T = np.zeros((N, N))
    for j in range(m):
        D = log.tau_diag[j]
        T[j * s:(j + 1) * s, j * s:(j + 1) * s] = 0.5 * (D + D.T)
        if j + 1 < m:
            T[(j + 1) * s:(j + 2) * s, j * s:(j + 1) * s] = log.tau_next[j]
            T[j * s:(j + 1) * s, (j + 1) * s:(j + 2) * s] = log.tau_next[j].T
    ab = np.zeros((s + 1, N))
    for d in range(s + 1):
        ab[d, : N - d] = np.diagonal(T, -d)
    return ab


def dense_T(log: LanczosLog, m: int) -> np.ndarray:
    """T_m as a dense symmetric matrix (from the same band)."""
    ab = band_T(log, m)
    s, N = log.s, log.s * m
    T = np.zeros((N, N))
    for d in range(s + 1):
        idx = np.arange(N - d)
        T[idx + d, idx] = ab[d, : N - d]
        T[idx, idx + d] = ab[d, : N - d]
    return T


def eig_T(log: LanczosLog, m: int):
    """Eigendecomposition T_m = Q Lambda Q^T exploiting the band (Sec. 3.2).

    LAPACK's band driver (via scipy.linalg.eig_banded) stands in for the
    paper's tridiagonalisation followed by a tridiagonal eigensolver; only
    eigenvalues and eigenvectors are used downstream.
    """
    lam, Q = sla.eig_banded(band_T(log, m), lower=True)
    return lam, Q


def cheap_residual(lam, Q, gamma, tau_next, s):
    """||R_m||_F from the eigenpairs of T_m (Prop. 3.1, Algorithm 3).

    a = Q^T E_1 gamma, so S_m = a a^T; W_m = Q^T E_m tau_{m+1,m}^T;
    ||R||^2 = 2 sum_i || e_i^T S_m D_i^{-1} W_m ||^2 with D_i = lambda_i I + Lambda.
    """
    a = Q[:s, :].T @ gamma            # (sm, s): rows a_i
    Wm = Q[-s:, :].T @ tau_next.T     # (sm, s)
    res = 0.0
    for i in range(lam.shape[0]):
        row = (a[i] @ a.T) / (lam[i] + lam)   # e_i^T S_m D_i^{-1}
        v = row @ Wm
        res += float(v @ v)
    return np.sqrt(2.0) * np.sqrt(res)


def residual_at(log: LanczosLog, m: int) -> float:
    """Relative residual ||R_m||_F / beta^2 (Alg. 1 step 6.3) for the space of dimension s*m."""
    lam, Q = eig_T(log, m)
    res = cheap_residual(lam, Q, log.gamma, log.tau_next[m - 1], log.s)
    return res / log.beta**2


@dataclass
class SolveResult:
    log: LanczosLog
    history: np.ndarray     # relative residual at m = 1..m_final (NaN where not checked)
    m: int
    converged: bool
    tol: float = 1e-8


def auto_trunc_eps(tol, norm_T, norm_J=None):
    """Truncation threshold of eq. 2.5 tied to the residual target (relative to ||C1|| ||C2||).

    The paper uses eps = 1e-12 with ||C||_F = 1 and tol = 1e-6.  Truncating the reduced solution
    by a tail of Frobenius norm eps moves A X + X B by at most (||A||_2 + ||B||_2) eps, so on
    operators with ||A|| ~ 1e5 a fixed 1e-12 alone would leave a residual ~1e-7.  The reading
    used here keeps the truncation's share at tol / 10:
        eps = min(1e-12, tol / (10 (||T_m||_2 + ||J_m||_2)))   (J_m = T_m for Lyapunov),
    with ||T_m||_2 (<= ||A||_2, close to it once the extreme Ritz values have converged) the
    largest |eigenvalue| of T_m.
    """
    nj = norm_T if norm_J is None else norm_J
    if not (norm_T + nj > 0) or not np.isfinite(norm_T + nj):
        return 1e-12
    return min(1e-12, tol / (10.0 * (norm_T + nj)))


def solve(A, C, tol=1e-8, maxit=1000, check_every=1, keep_basis=False) -> SolveResult:
    """Algorithm 1 with the standard block Krylov space, steps 1-7.

    The convergence test is applied at every ``check_every``-th space
    dimension (the paper's d, Sec. 6), and at the first m with relative
    residual <= tol the iteration stops.
    """
    V1, log = start(C, keep_basis)
    Vprev, Vcur = None, V1
    hist = []
    converged = False
    m = 0
    for j in range(1, maxit + 1):
        Vnext, tp, td, tn = lanczos_step(A, Vprev, Vcur)
        log.tau_prev.append(tp)
        log.tau_diag.append(td)
        log.tau_next.append(tn)
        if log.basis is not None:
            log.basis.append(Vnext)
        Vprev, Vcur = Vcur, Vnext
        m = j
        if j % check_every == 0:
            rel = residual_at(log, j)
            hist.append(rel)
            if rel <= tol:
                converged = True
                break
        else:
            hist.append(np.nan)
    return SolveResult(log=log, history=np.array(hist), m=m, converged=converged, tol=tol)


def truncated_factor(log: LanczosLog, m: int, trunc_eps: float | None = None, tol: float | None = None):
    """Low-rank factor of the reduced solution, truncated in the eigenbasis of T_m.

    Y~ = -(e_i^T S e_j / (lambda_i + lambda_j))_{ij} (eq. 3.2); its eigenvalues
    sigma (non-increasing) are truncated so that the discarded tail has
    Frobenius norm <= eps (eq. 2.5, applied to Y~ as in Sec. 3.2), with
    eps = trunc_eps * beta^2 (trunc_eps None: auto_trunc_eps(tol, ||T_m||));
    negative sigma (rounding) are never kept.
    Returns M = Q_m Ycheck (s*m x t) such that Y_m ~= M M^T, and the kept sigma.
    """
    s = log.s
    lam, Q = eig_T(log, m)
    if trunc_eps is None:
        trunc_eps = auto_trunc_eps(tol, float(np.max(np.abs(lam))))
    a = Q[:s, :].T @ log.gamma
    Yt = -(a @ a.T) / (lam[:, None] + lam[None, :])
    sig, Wv = np.linalg.eigh(Yt)
    order = np.argsort(sig)[::-1]
    sig, Wv = sig[order], Wv[:, order]
    eps_abs = trunc_eps * log.beta**2
    npos = int(np.sum(sig > 0))
    # tail[t] = ||sigma_{t+1:}||_2 with t kept values
    tail = np.sqrt(np.concatenate([np.cumsum((sig**2)[::-1])[::-1], [0.0]]))
    t = int(np.argmax(tail <= eps_abs))
    t = min(t, npos)
    Ycheck = Wv[:, :t] * np.sqrt(sig[:t])
    return Q @ Ycheck, sig[:t]


def regenerate_basis(A, C, log: LanczosLog, m: int):
    """Second Lanczos pass (Sec. 3.3): yields V_1..V_m from the stored coefficients.

    V_{j+1} = (A V_j - V_j tau_{jj} - V_{j-1} tau_{j-1,j}) tau_{j+1,j}^{-1},
    with the raw (non-symmetrised) coefficients, and V_1 from the same QR of C.
    """
    V1, _ = qr_pos(np.asarray(C, dtype=np.float64))
    Vprev, Vcur = None, V1
    for j in range(1, m + 1):
        yield Vcur
        if j == m:
            break
        W = A @ Vcur - Vcur @ log.tau_diag[j - 1]
        if Vprev is not None:
            W = W - Vprev @ log.tau_prev[j - 1]
        # right-multiplication by the inverse of the upper-triangular tau_{j+1,j}
        Vnext = sla.solve_triangular(log.tau_next[j - 1], W.T, trans="T", lower=False).T
        Vprev, Vcur = Vcur, Vnext


def factor(A, C, res: SolveResult, trunc_eps: float | None = None, two_pass: bool = True):
    """Alg. 1 steps 8-9: Z_m = V_m (Q_m Ycheck), by the two-pass device or the stored basis.
    trunc_eps None: the tolerance-consistent threshold of auto_trunc_eps with the solve's tol."""
    s, m = res.log.s, res.m
    M, sig = truncated_factor(res.log, m, trunc_eps, res.tol)
    n = C.shape[0]
    Z = np.zeros((n, M.shape[1]))
    if two_pass:
        for j, Vj in enumerate(regenerate_basis(A, C, res.log, m)):
            Z += Vj @ M[j * s:(j + 1) * s, :]
    else:
        if res.log.basis is None:
            raise ValueError("stored-basis factor needs keep_basis=True")
        for j in range(m):
            Z += res.log.basis[j] @ M[j * s:(j + 1) * s, :]
    return Z, sig
