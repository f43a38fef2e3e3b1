"""FP64 oracle of the inner solves with A for the extended Krylov space (Sec. 4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper applies A^{-1} to the second half of each basis block with a direct solver (the
cost of those solves is reported separately in Sec. 6).  The CUDA path replaces the direct
solver by preconditioned conjugate gradients on M = -A, which is symmetric positive definite
since A is symmetric negative definite.  This module restates, from their published
definitions:

  * conjugate gradients with a preconditioner P ~ M^{-1} (Hestenes and Stiefel, 1952), in its
    textbook form: one product with M, one application of P and two inner products per
    iteration, stopped at ||b - M x|| <= tol ||b|| on the recursively updated residual;
  * Jacobi scaling, P r = r / diag(M);
  * the zero-fill incomplete Cholesky factorisation IC(0) (Meijerink and van der Vorst, 1977):
    the lower-triangular L with the sparsity pattern of tril(M) such that (L L^T)_{ik} = M_{ik}
    for every (i, k) in that pattern, computed row by row:
        L_ik = (M_ik - sum_{j < k} L_ij L_kj) / L_kk   for k < i in the pattern of row i,
        L_ii = sqrt(M_ii - sum_{j < i} L_ij^2),
    with the sums over columns j in the patterns of both rows; P r = (L L^T)^{-1} r by a
    forward and a backward triangular solve;
  * the modified factorisation MIC(0) (Gustafsson, 1978): the same pattern, but each update of
    the elimination that falls outside the pattern is subtracted from the diagonals of its row
    and its column instead of being dropped, so that L L^T has the row sums of M,
    (L L^T) 1 = M 1;
  * the factorised sparse approximate inverse FSAI (Kolotilina and Yeremin, 1993): G lower
    triangular on a chosen pattern, row i from the local system M[J_i, J_i] g = e_i on its
    pattern J_i, scaled so that (G M G^T)_ii = 1; P r = G^T (G r), products only.

Plain Python loops over the rows: for the small grids of the tests only.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class IC0Breakdown(ArithmeticError):
    """A non-positive pivot: IC(0) does not exist for this matrix."""


def ic0(M) -> sp.csr_matrix:
    """IC(0) factor L of the symmetric positive definite sparse matrix M (CSR, lower triangle
    with the diagonal; only tril(M) is read)."""
    Ml = sp.csr_matrix(sp.tril(M))
    Ml.sort_indices()
    n = Ml.shape[0]
    rows: list[dict[int, float]] = []  # row i of L as {column: value}
    for i in range(n):
        lo, hi = Ml.indptr[i], Ml.indptr[i + 1]
        cols, vals = Ml.indices[lo:hi], Ml.data[lo:hi]
        row: dict[int, float] = {}
        diag = 0.0
        for c, v in zip(cols, vals):
            c = int(c)
            if c == i:
                diag = float(v)
                continue
            # L_ic = (M_ic - sum_{j < c} L_ij L_cj) / L_cc, columns j already in row i
            rk = rows[c]
            acc = float(v)
            for j, lij in row.items():
                if j < c:
                    lkj = rk.get(j)
                    if lkj is not None:
                        acc -= lij * lkj
            row[c] = acc / rk[c]
        d = diag - sum(x * x for x in row.values())
        if not d > 0.0:
            raise IC0Breakdown(f"pivot {d} at row {i}")
        row[i] = float(np.sqrt(d))
        rows.append(row)
    indptr = np.zeros(n + 1, dtype=np.int64)
    indices, data = [], []
    for i, row in enumerate(rows):
        for c in sorted(row):
            indices.append(c)
            data.append(row[c])
        indptr[i + 1] = len(indices)
    return sp.csr_matrix((np.array(data), np.array(indices, dtype=np.int64), indptr), shape=(n, n))


def mic0(M) -> sp.csr_matrix:
    """MIC(0) factor L of the symmetric positive definite sparse matrix M: right-looking
    elimination on the pattern of tril(M); the update l_ik l_jk of an entry (i, j) outside the
    pattern is subtracted from a_ii and a_jj."""
    Ml = sp.csc_matrix(sp.tril(M))
    Ml.sort_indices()
    n = Ml.shape[0]
    # working lower triangle by columns: col[k] = {row: value}, rows >= k
    col = []
    for k in range(n):
        lo, hi = Ml.indptr[k], Ml.indptr[k + 1]
        col.append({int(r): float(v) for r, v in zip(Ml.indices[lo:hi], Ml.data[lo:hi])})
    diag = np.array([col[k].get(k, 0.0) for k in range(n)])
    L_cols = []
    for k in range(n):
        d = diag[k]
        if not d > 0.0:
            raise IC0Breakdown(f"pivot {d} at row {k}")
        lkk = float(np.sqrt(d))
        below = sorted(r for r in col[k] if r > k)
        lk = {r: col[k][r] / lkk for r in below}
        L_cols.append((lkk, lk))
        # Schur complement on the pattern; updates outside it go to both diagonals
        for a, i in enumerate(below):
            li = lk[i]
            diag[i] -= li * li
            for j in below[:a]:
                u = li * lk[j]  # entry (i, j), i > j > k
                if i in col[j]:
                    col[j][i] -= u
                else:
                    diag[i] -= u
                    diag[j] -= u
    rows_i, cols_i, vals = [], [], []
    for k, (lkk, lk) in enumerate(L_cols):
        rows_i.append(k); cols_i.append(k); vals.append(lkk)
        for r, v in lk.items():
            rows_i.append(r); cols_i.append(k); vals.append(v)
    return sp.csr_matrix((vals, (rows_i, cols_i)), shape=(n, n))


def fsai(M, patterns) -> sp.csr_matrix:
    """FSAI factor G of the SPD matrix M; ``patterns[i]`` lists the columns j <= i of row i
    (it must contain i)."""
    M = sp.csr_matrix(M)
    n = M.shape[0]
    rows, cols, vals = [], [], []
    for i in range(n):
        J = sorted(set(int(j) for j in patterns[i]))
        if i not in J or J[-1] != i:
            raise ValueError(f"row {i}: the pattern must end at the diagonal")
        MJ = M[J][:, J].toarray()
        e = np.zeros(len(J))
        e[-1] = 1.0
        g = np.linalg.solve(MJ, e)
        if not g[-1] > 0.0:
            raise ArithmeticError(f"row {i}: non-positive FSAI pivot")
        g /= np.sqrt(g[-1])
        rows += [i] * len(J)
        cols += J
        vals += list(g)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def grid_lower_patterns(k: int, reach: int):
    """For a k x k grid (x fastest): row i's pattern is every node j <= i within `reach` cells
    of i in both directions (reach 1: the lower half of the 3 x 3 neighbourhood)."""
    pats = []
    for i in range(k * k):
        xi, yi = i % k, i // k
        J = [y * k + x for y in range(max(0, yi - reach), yi + 1)
             for x in range(max(0, xi - reach), min(k, xi + reach + 1)) if y * k + x <= i]
        pats.append(J)
    return pats


def fsai_prec(G):
    """P r = G^T (G r)."""
    G = sp.csr_matrix(G)
    Gt = sp.csr_matrix(G.T)
    return lambda r: Gt @ (G @ r)


def jacobi_prec(M):
    """P r = r / diag(M)."""
    d = np.asarray(M.diagonal(), dtype=np.float64)
    return lambda r: r / d


def ic0_prec(L):
    """P r = (L L^T)^{-1} r: forward solve with L, backward solve with L^T."""
    L = sp.csr_matrix(L)
    Lt = sp.csr_matrix(L.T)

    def apply(r):
        y = spla.spsolve_triangular(L, r, lower=True)
        return spla.spsolve_triangular(Lt, y, lower=False)

    return apply


@dataclass
class CGResult:
    x: np.ndarray
    iterations: int
    converged: bool
    residuals: np.ndarray  # ||r_k|| / ||b||, k = 0 .. iterations


def pcg(M, b, prec=None, tol: float = 1e-10, maxit: int = 10000) -> CGResult:
    """Preconditioned conjugate gradients for M x = b from x = 0."""
    b = np.asarray(b, dtype=np.float64)
    P = prec if prec is not None else (lambda r: r)
    x = np.zeros_like(b)
    r = b.copy()
    nb = float(np.linalg.norm(b))
    hist = [1.0 if nb > 0 else 0.0]
    if nb == 0.0:
        return CGResult(x, 0, True, np.array(hist))
    z = P(r)
    p = z.copy()
    rz = float(r @ z)
    for it in range(1, maxit + 1):
        q = M @ p
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        rel = float(np.linalg.norm(r)) / nb
        hist.append(rel)
        if rel <= tol:
            return CGResult(x, it, True, np.array(hist))
        z = P(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return CGResult(x, maxit, False, np.array(hist))
