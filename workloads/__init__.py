"""Seeded synthetic problem generators shared by the oracle, the tests and the bench.

This module defines *problems* only: sparse symmetric negative definite operators
and tall right-hand sides.  It holds none of the solver's arithmetic (no Krylov
basis, no projection, no residual), so that the CPU oracle and the CUDA path can
both consume identical inputs without sharing any of the method.

Discretisation conventions (zero Dirichlet boundary, lexicographic ordering with
x fastest, mesh width h = 1/(k+1), A = -(1/h^2) * SPD stencil matrix) follow the
finite-difference operators of the paper's experiments (Section 6).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Problem",
    "laplacian_2d",
    "laplacian_3d",
    "var_coeff_diffusion",
    "gaussian_field",
    "fd_operator",
    "paper_ex61_operator",
    "paper_ex64_operator_B",
    "paper_rand_rhs",
    "rhs",
    "random_snd_dense",
    "fe_mass_stiffness_2d",
    "batched_instances",
    "config_c1",
    "config_c2",
    "config_c3",
    "config_c4",
]


@dataclass
class Problem:
    """A Lyapunov (B is None) or Sylvester problem A X + X B + C1 C2^T = 0."""

    name: str
    A: sp.csr_matrix
    C1: np.ndarray
    B: sp.csr_matrix | None = None
    C2: np.ndarray | None = None
    tol: float = 1e-8
    maxit: int = 1000

    @property
    def s(self) -> int:
        return int(self.C1.shape[1])


def _csr(m: sp.spmatrix, dtype=np.float64) -> sp.csr_matrix:
    m = sp.csr_matrix(m, dtype=np.float64)
    m.sum_duplicates()
    m.sort_indices()
    if dtype == np.float32:
        # values rounded to fp32 and promoted back: both sides then see the same A
        m.data = m.data.astype(np.float32).astype(np.float64)
    return m


def _tridiag_spd(k: int) -> sp.csr_matrix:
    e = np.ones(k)
    return sp.diags([-e[:-1], 2.0 * e, -e[:-1]], [-1, 0, 1], format="csr")


def laplacian_2d(k: int, shift: float = 0.0) -> sp.csr_matrix:
    """A = -(1/h^2)(T(x)I + I(x)T) - shift*I on a k x k grid, h = 1/(k+1)."""
    h2 = float(k + 1) ** 2
    T = _tridiag_spd(k)
    I = sp.identity(k, format="csr")
    A = -h2 * (sp.kron(I, T) + sp.kron(T, I))
    if shift:
        A = A - shift * sp.identity(k * k)
    return _csr(A)


def laplacian_3d(k: int) -> sp.csr_matrix:
    """A = -(1/h^2)(T(x)I(x)I + I(x)T(x)I + I(x)I(x)T) on a k^3 grid, h = 1/(k+1)."""
    h2 = float(k + 1) ** 2
    T = _tridiag_spd(k)
    I = sp.identity(k, format="csr")
    A = -h2 * (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I))
    return _csr(A)


def var_coeff_diffusion(kappa: np.ndarray, dtype=np.float64) -> sp.csr_matrix:
    """A = -div(kappa grad u) by the 5/7-point finite-volume stencil.

    ``kappa`` holds nodal coefficients on a k x k (or k x k x k) grid, indexed
    [z][y][x].  The coefficient on the face between two nodes is the harmonic
    mean of the nodal values; a face on the boundary uses the interior node's
    value.  Off-diagonals are +kappa_f/h^2, the diagonal is -sum(kappa_f)/h^2.
    """
    kappa = np.asarray(kappa, dtype=np.float64)
    shape = kappa.shape
    k = shape[0]
    assert all(d == k for d in shape)
    h2 = float(k + 1) ** 2
    n = kappa.size
    idx = np.arange(n).reshape(shape)
    kap = kappa
    rows, cols, vals = [], [], []
    diag = np.zeros(shape)
    for axis in range(kappa.ndim):
        # axis 0 of the array is the slowest coordinate; x is the last axis
        sl_lo = [slice(None)] * kappa.ndim
        sl_hi = [slice(None)] * kappa.ndim
        sl_lo[axis] = slice(0, k - 1)
        sl_hi[axis] = slice(1, k)
        a = kap[tuple(sl_lo)]
        b = kap[tuple(sl_hi)]
        face = 2.0 * a * b / (a + b)
        i_lo = idx[tuple(sl_lo)].ravel()
        i_hi = idx[tuple(sl_hi)].ravel()
        f = face.ravel() * h2
        rows += [i_lo, i_hi]
        cols += [i_hi, i_lo]
        vals += [f, f]
        d_lo = np.zeros(shape)
        d_lo[tuple(sl_lo)] += face
        d_lo[tuple(sl_hi)] += face
        # boundary faces at both ends of this axis use the nodal value
        first = [slice(None)] * kappa.ndim
        last = [slice(None)] * kappa.ndim
        first[axis] = 0
        last[axis] = k - 1
        d_lo[tuple(first)] += kap[tuple(first)]
        d_lo[tuple(last)] += kap[tuple(last)]
        diag += d_lo
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(-diag.ravel() * h2)
    A = sp.csr_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)
    )
    return _csr(A, dtype)


def gaussian_field(k: int, ndim: int, seed: int, corr_len: float | None = None) -> np.ndarray:
    """Unit-variance Gaussian field on a k^ndim grid.

    ``corr_len=None`` gives iid N(0,1) values.  Otherwise white noise is
    convolved with a Gaussian kernel of that correlation length (in cells) by
    FFT on a periodic grid padded by 4*corr_len, cropped, and rescaled to unit
    sample variance.
    """
    rng = np.random.default_rng(seed)
    if corr_len is None:
        return rng.standard_normal((k,) * ndim)
    pad = int(4 * corr_len)
    m = k + pad
    noise = rng.standard_normal((m,) * ndim)
    freqs = [np.fft.fftfreq(m) for _ in range(ndim)]
    grids = np.meshgrid(*freqs, indexing="ij")
    w2 = sum(g**2 for g in grids)
    # Fourier transform of exp(-r^2 / (2 l^2)) up to a constant
    kernel_hat = np.exp(-2.0 * (np.pi**2) * (corr_len**2) * w2)
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * kernel_hat))
    field = field[tuple(slice(0, k) for _ in range(ndim))]
    field = (field - field.mean()) / field.std()
    return field


def fd_operator(k: int, ax, by) -> sp.csr_matrix:
    """Centred differences of (a(x,y) u_x)_x + (b(x,y) u_y)_y on the unit square.

    Zero Dirichlet boundary, h = 1/(k+1), coefficients evaluated at the
    cell-face midpoints; ``ax`` and ``by`` are vectorised callables.
    """
    h = 1.0 / (k + 1)
    xs = h * np.arange(1, k + 1)
    n = k * k
    idx = np.arange(n).reshape(k, k)  # [y][x]
    X, Y = np.meshgrid(xs, xs, indexing="xy")  # X[j, i] = x_i, Y[j, i] = y_j
    aE = ax(X + h / 2, Y)
    aW = ax(X - h / 2, Y)
    bN = by(X, Y + h / 2)
    bS = by(X, Y - h / 2)
    h2 = 1.0 / h**2
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [-(aE + aW + bN + bS).ravel() * h2]
    rows.append(idx[:, :-1].ravel()); cols.append(idx[:, 1:].ravel()); vals.append(aE[:, :-1].ravel() * h2)
    rows.append(idx[:, 1:].ravel()); cols.append(idx[:, :-1].ravel()); vals.append(aW[:, 1:].ravel() * h2)
    rows.append(idx[:-1, :].ravel()); cols.append(idx[1:, :].ravel()); vals.append(bN[:-1, :].ravel() * h2)
    rows.append(idx[1:, :].ravel()); cols.append(idx[:-1, :].ravel()); vals.append(bS[1:, :].ravel() * h2)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return _csr(A)


def paper_ex61_operator(k: int = 148) -> sp.csr_matrix:
    """(e^{-xy} u_x)_x + (e^{xy} u_y)_y (Section 6, Examples 6.1 and 6.4; n = 21904 / 16384)."""
    return fd_operator(k, lambda x, y: np.exp(-x * y), lambda x, y: np.exp(x * y))


def paper_ex64_operator_B(k: int = 128) -> sp.csr_matrix:
    """(sin(xy) u_x)_x + (cos(xy) u_y)_y (Section 6, Example 6.4; n = 16384)."""
    return fd_operator(k, lambda x, y: np.sin(x * y), lambda x, y: np.cos(x * y))


def paper_rand_rhs(n: int, s: int, seed: int) -> np.ndarray:
    """C = rand(n, s) / ||rand(n, s)||_F as in the paper's experiments (uniform on (0,1))."""
    C = np.random.default_rng(seed).uniform(0.0, 1.0, (n, s))
    return np.ascontiguousarray(C / np.linalg.norm(C, "fro"))


def rhs(n: int, s: int, seed: int) -> np.ndarray:
    """Tall right-hand side, iid N(0,1), fp64, row-major n x s."""
    return np.ascontiguousarray(np.random.default_rng(seed).standard_normal((n, s)))


def random_snd_dense(n: int, seed: int, lam_min: float = 1.0, lam_max: float = 100.0) -> np.ndarray:
    """Dense symmetric negative definite matrix with a log-uniform spectrum."""
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = -np.exp(rng.uniform(np.log(lam_min), np.log(lam_max), n))
    A = (Qm * lam) @ Qm.T
    return 0.5 * (A + A.T)


def fe_mass_stiffness_2d(k: int, kappa=None):
    """Bilinear (Q1) finite elements on the unit square with k x k interior nodes and zero
    Dirichlet values: the mass matrix E (symmetric positive definite) and A = -K, K the
    stiffness matrix of -div(kappa grad u) (symmetric positive definite), so that A is
    symmetric negative definite.  ``kappa`` (k+1 x k+1 element values, default 1) gives
    variable coefficients.  The generalised Lyapunov equation A X E + E X A + C C^T = 0 of the
    paper's example with a mass matrix uses this pair as a synthetic stand-in."""
    h = 1.0 / (k + 1)
    ne = k + 1
    kap = np.ones((ne, ne)) if kappa is None else np.asarray(kappa, dtype=np.float64)
    # element matrices on a square of side h, local nodes (0,0), (1,0), (0,1), (1,1)
    m1 = h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    k1 = 1.0 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
    Me = np.kron(m1, m1)
    Ke = np.kron(k1, m1) + np.kron(m1, k1)
    rows, cols, mv, kv = [], [], [], []
    for ey in range(ne):
        for ex in range(ne):
            loc = []
            for dy in (0, 1):
                for dx in (0, 1):
                    gx, gy = ex + dx - 1, ey + dy - 1  # interior node indices, -1 / k on the boundary
                    loc.append(gy * k + gx if 0 <= gx < k and 0 <= gy < k else -1)
            # np.kron(a, b) puts the index of a first: local order (dy, dx) matches (y-major, x-minor)
            for a in range(4):
                for b in range(4):
                    if loc[a] >= 0 and loc[b] >= 0:
                        rows.append(loc[a]); cols.append(loc[b])
                        mv.append(Me[a, b]); kv.append(kap[ey, ex] * Ke[a, b])
    n = k * k
    E = sp.csr_matrix((mv, (rows, cols)), shape=(n, n))
    K = sp.csr_matrix((kv, (rows, cols)), shape=(n, n))
    return _csr(-K), _csr(E)


def batched_instances(count: int = 256, seed: int = 0, kmin: int = 64, kmax: int = 512):
    """(k_i, d_i, s_i) for the batched Lyapunov workload.

    k uniform in [kmin, kmax], shift d uniform in [0, 10], block size s in {1, 2, 4};
    instance i is A_i = -(2D Laplacian on k_i x k_i) - d_i I with C_i = rhs(k_i^2, s_i, seed + 1 + i).
    """
    rng = np.random.default_rng(seed)
    ks = rng.integers(kmin, kmax + 1, size=count)
    ds = rng.uniform(0.0, 10.0, size=count)
    ss = rng.choice(np.array([1, 2, 4]), size=count)
    return [(int(k), float(d), int(s)) for k, d, s in zip(ks, ds, ss)]


def config_c4(seed: int = 0, count: int = 256, kmin: int = 64, kmax: int = 512) -> list:
    """Batched Lyapunov: instance i is A_i = -(2D Laplacian on k_i x k_i) - d_i I with
    (k_i, d_i, s_i) from batched_instances, values rounded to fp32 (both the GPU's fp32 operator
    and the fp64 oracle see the same A_i), C_i = rhs(k_i^2, s_i, seed + 1 + i), tol 1e-8."""
    out = []
    for i, (k, d, s) in enumerate(batched_instances(count, seed, kmin, kmax)):
        A = laplacian_2d(k, shift=d)
        A.data = A.data.astype(np.float32).astype(np.float64)
        out.append(Problem(f"lyap_lap2d_{k}_d{d:.3f}_s{s}", A, rhs(k * k, s, seed + 1 + i), tol=1e-8, maxit=1000))
    return out


def config_c1(seed: int = 0) -> Problem:
    """Lyapunov, 2D 5-point Laplacian on 50 x 50 (n = 2500), s = 1, tol 1e-8."""
    A = laplacian_2d(50)
    return Problem("lyap_lap2d_50_s1", A, rhs(A.shape[0], 1, seed), tol=1e-8, maxit=1000)


def config_c2(seed: int = 0, k: int = 100, s: int = 4) -> Problem:
    """Lyapunov, 3D 7-point Laplacian on 100^3 (n = 1e6), s = 4, tol 1e-8, max 400 its."""
    A = laplacian_3d(k)
    return Problem(f"lyap_lap3d_{k}_s{s}", A, rhs(A.shape[0], s, seed), tol=1e-8, maxit=400)


def config_c3(seed: int = 0, ka: int = 80, kb: int = 500, s: int = 2, sigma: float = 1.0) -> Problem:
    """Sylvester: A = 3D variable-coefficient diffusion on ka^3 (log-normal, fp32 values),
    B = 2D 5-point Laplacian on kb x kb, s = 2, tol 1e-8."""
    kappa = np.exp(sigma * gaussian_field(ka, 3, seed=1000 + seed))
    A = var_coeff_diffusion(kappa, dtype=np.float32)
    B = laplacian_2d(kb)
    C1 = rhs(A.shape[0], s, 2 * seed + 1)
    C2 = rhs(B.shape[0], s, 2 * seed + 2)
    return Problem(f"sylv_vc3d_{ka}_lap2d_{kb}_s{s}", A, C1, B, C2, tol=1e-8, maxit=2000)
