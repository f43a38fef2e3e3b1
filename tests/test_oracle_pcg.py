"""Pins of the inner-solve oracle (oracle/pcg.py): conjugate gradients, Jacobi and IC(0)
preconditioning for M = -A, checked against facts that do not depend on the code under test.

  * IC(0) of a tridiagonal matrix has no fill to drop, so it is the exact Cholesky factor.
  * On the 5-point Laplacian, L L^T equals M on the sparsity pattern of M (the definition)
    and differs from it off the pattern (IC(0) is not the exact factor there).  Rows of that
    pattern share no earlier column, so the same check on the 9-point stencil, whose rows do,
    pins the cross terms of the factorisation.
  * The same IC(0) pivots obey d_k = 4 - 1/d_{k-1} - 1/d_{k-nx} in the interior (stencil 4,
    -1), whose fixed point is 2 + sqrt(2): far from the first rows the pivots approach it.
  * Conjugate gradients in exact arithmetic end in at most as many steps as M has distinct
    eigenvalues: a diagonal matrix with three distinct values is solved in three.
  * On the variable-coefficient diffusion operator both preconditioned solves reach the
    tolerance, agree with a direct solve, and IC(0) needs fewer iterations than Jacobi.
  * MIC(0) keeps the row sums, (L L^T) 1 = M 1, and agrees with M off the diagonal on the
    pattern.  On the 5-point stencil its pivots obey d = 4 - 2/d_west - 2/d_south, so every
    pivot is at least 2 and the interior ones approach the double root d = 2 of d = 4 - 4/d.
    It needs fewer iterations than IC(0) on the variable-coefficient operator.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as wl
from oracle import pcg


def test_ic0_of_tridiagonal_is_exact_cholesky():
    rng = np.random.default_rng(3)
    n = 40
    off = -rng.uniform(0.5, 1.5, n - 1)
    main = 2.5 + rng.uniform(0.0, 1.0, n)  # diagonally dominant, so SPD
    M = sp.diags([off, main, off], [-1, 0, 1], format="csr")
    L = pcg.ic0(M).toarray()
    Lc = np.linalg.cholesky(M.toarray())
    assert np.max(np.abs(L - Lc)) <= 1e-14 * np.max(np.abs(Lc))


def test_ic0_matches_on_pattern_and_drops_fill():
    k = 12
    M = -wl.laplacian_2d(k) / float(k + 1) ** 2  # the stencil (4, -1, -1, -1, -1)
    L = pcg.ic0(M)
    LLt = (L @ L.T).toarray()
    Md = M.toarray()
    pattern = Md != 0.0
    assert np.max(np.abs((LLt - Md)[pattern])) <= 1e-13
    # fill of the exact factor, dropped by IC(0): L L^T has entries outside the pattern
    assert np.max(np.abs(LLt[~pattern])) > 1e-3
    # L itself keeps the pattern of tril(M)
    Lp = L.toarray() != 0.0
    assert not np.any(Lp & ~np.tril(pattern))


def test_ic0_matches_on_pattern_with_shared_columns():
    k = 10
    # 9-point stencil: 8 on the diagonal, -1 for each of the eight neighbours (an M-matrix)
    T = sp.diags([1.0, 1.0, 1.0], [-1, 0, 1], shape=(k, k))
    N = sp.kron(T, T, format="csr")  # the 3 x 3 neighbourhood of every node, itself included
    M = sp.csr_matrix(9.0 * sp.identity(k * k) - N)
    Md = M.toarray()
    assert np.all(np.linalg.eigvalsh(Md) > 0)
    L = pcg.ic0(M)
    LLt = (L @ L.T).toarray()
    pattern = Md != 0.0
    assert np.max(np.abs((LLt - Md)[pattern])) <= 1e-13
    assert np.max(np.abs(LLt[~pattern])) > 1e-3


def test_ic0_pivots_approach_closed_form_fixed_point():
    k = 48
    M = -wl.laplacian_2d(k) / float(k + 1) ** 2
    d = pcg.ic0(M).diagonal() ** 2
    grid = d.reshape(k, k)
    target = 2.0 + np.sqrt(2.0)
    # deep rows, interior columns: converged to the fixed point of d = 4 - 2/d
    interior = grid[k - 8:k - 1, k // 2 - 4:k // 2 + 4]
    assert np.max(np.abs(interior - target)) < 2e-3
    # the first pivot is the diagonal itself
    assert abs(d[0] - 4.0) < 1e-14


def test_cg_terminates_in_number_of_distinct_eigenvalues():
    vals = np.repeat([1.0, 3.0, 10.0], [7, 5, 4])
    M = sp.diags(vals, 0, format="csr")
    b = np.random.default_rng(0).standard_normal(vals.size)
    res = pcg.pcg(M, b, tol=1e-12, maxit=50)
    assert res.converged and res.iterations == 3
    assert np.allclose(res.x, b / vals, rtol=1e-12, atol=0)


def test_jacobi_cg_on_a_diagonal_matrix_is_one_step():
    vals = np.linspace(1.0, 50.0, 30)
    M = sp.diags(vals, 0, format="csr")
    b = np.random.default_rng(1).standard_normal(30)
    res = pcg.pcg(M, b, prec=pcg.jacobi_prec(M), tol=1e-14, maxit=5)
    assert res.converged and res.iterations == 1


@pytest.mark.parametrize("k", [32])
def test_ic0_beats_jacobi_on_variable_coefficients(k):
    kappa = np.exp(1.5 * wl.gaussian_field(k, 2, seed=5, corr_len=4.0))
    M = -wl.var_coeff_diffusion(kappa)
    b = wl.rhs(k * k, 1, seed=7)[:, 0]
    x_ref = spla.spsolve(sp.csc_matrix(M), b)
    rj = pcg.pcg(M, b, prec=pcg.jacobi_prec(M), tol=1e-10, maxit=5000)
    ri = pcg.pcg(M, b, prec=pcg.ic0_prec(pcg.ic0(M)), tol=1e-10, maxit=5000)
    for r in (rj, ri):
        assert r.converged
        assert np.linalg.norm(M @ r.x - b) <= 1e-9 * np.linalg.norm(b)
        assert np.linalg.norm(r.x - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
    assert ri.iterations < 0.7 * rj.iterations


def test_mic0_keeps_row_sums_and_pattern():
    k = 24
    kappa = np.exp(1.5 * wl.gaussian_field(k, 2, seed=5, corr_len=4.0))
    M = -wl.var_coeff_diffusion(kappa)
    L = pcg.mic0(M)
    one = np.ones(k * k)
    rs = M @ one
    assert np.max(np.abs(L @ (L.T @ one) - rs)) <= 1e-13 * np.max(np.abs(M.diagonal()))
    Md = M.toarray()
    LLt = (L @ L.T).toarray()
    off = (Md != 0.0) & ~np.eye(k * k, dtype=bool)
    assert np.max(np.abs((LLt - Md)[off])) <= 1e-13 * np.max(np.abs(Md))
    # the diagonal is where it differs from IC(0): the dropped fill lands there
    assert np.max(np.abs(np.diag(LLt) - np.diag(Md))) > 1e-3 * np.max(np.abs(Md))


def test_mic0_pivots_on_the_laplacian():
    k = 48
    M = -wl.laplacian_2d(k) / float(k + 1) ** 2
    d = pcg.mic0(M).diagonal() ** 2
    assert d.min() >= 2.0 - 1e-12
    assert abs(d[0] - 4.0) < 1e-14
    deep = d.reshape(k, k)[k - 8:k - 1, k // 2 - 4:k // 2 + 4]
    assert np.max(deep) < 2.1  # IC(0) pivots there are near 2 + sqrt(2)


def test_mic0_beats_ic0_on_variable_coefficients():
    k = 64
    kappa = np.exp(1.5 * wl.gaussian_field(k, 2, seed=1000, corr_len=2.0))
    M = -wl.var_coeff_diffusion(kappa)
    b = wl.rhs(k * k, 1, seed=7)[:, 0]
    ri = pcg.pcg(M, b, prec=pcg.ic0_prec(pcg.ic0(M)), tol=1e-8, maxit=5000)
    rm = pcg.pcg(M, b, prec=pcg.ic0_prec(pcg.mic0(M)), tol=1e-8, maxit=5000)
    assert ri.converged and rm.converged
    assert rm.iterations < 0.8 * ri.iterations


def test_fsai_on_the_full_lower_pattern_is_the_inverse_factor():
    rng = np.random.default_rng(8)
    n = 12
    B = rng.standard_normal((n, n))
    M = sp.csr_matrix(B @ B.T + n * np.eye(n))
    G = pcg.fsai(M, [list(range(i + 1)) for i in range(n)])
    # G^T G = M^{-1}: G is the inverse of the Cholesky factor of M
    assert np.allclose((G.T @ G).toarray(), np.linalg.inv(M.toarray()), rtol=0, atol=1e-12)


def test_fsai_scaling_and_pattern_growth():
    k = 24
    kappa = np.exp(1.5 * wl.gaussian_field(k, 2, seed=5, corr_len=4.0))
    M = -wl.var_coeff_diffusion(kappa)
    b = wl.rhs(k * k, 1, seed=7)[:, 0]
    its = []
    for reach in (1, 2):
        G = pcg.fsai(M, pcg.grid_lower_patterns(k, reach))
        d = (G @ M @ G.T).diagonal()
        assert np.max(np.abs(d - 1.0)) <= 1e-12
        assert np.all(G.diagonal() > 0)
        its.append(pcg.pcg(M, b, prec=pcg.fsai_prec(G), tol=1e-8).iterations)
    jac = pcg.pcg(M, b, prec=pcg.jacobi_prec(M), tol=1e-8).iterations
    assert its[1] < its[0] < jac
