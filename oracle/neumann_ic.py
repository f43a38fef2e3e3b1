"""FP64 oracle of the products-only preconditioners for the inner solves of the extended Krylov
method (Sec. 4 applies A^{-1} by direct solves; the iterative solves and their preconditioners
are additions, see oracle/pcg.py).

TEST INFRASTRUCTURE ONLY (see the package docstring).

M = -A is symmetric positive definite, from a 5-point stencil on an nx x ny grid (x fastest).
Its IC(0) factor L = D + N (Meijerink and van der Vorst, 1977; oracle/pcg.ic0) has the diagonal
D = diag(d) and two strictly lower entries per row, the west one lw_i = L_{i,i-1} and the south
one ls_i = L_{i,i-nx} (zero where the neighbour is outside the grid).

Truncated Neumann series.  With T = -D^{-1} N (strictly lower triangular, so nilpotent)
    L^{-1} = (I - T)^{-1} D^{-1} = sum_{t >= 0} T^t D^{-1},
and keeping the terms t = 0..q gives the lower-triangular
    B_q = sum_{t=0}^{q} T^t D^{-1},      B_q L = I - T^{q+1},
whose diagonal is 1/d > 0.  The preconditioner is P_q = B_q^T B_q ~ (L L^T)^{-1}: symmetric
positive definite by construction, applied with 2q sparse products and no triangular solve.

Learned values.  A network (oracle/learned_factor: the stencil row over its diagonal as 5
input channels, three 3x3 convolutions 5 -> 16 -> 16 -> 3) maps the operator to corrections
y = (y0, y1, y2) of the IC(0) values,
    d = d0 exp(y0),   lw = lw0 (1 + y1),   ls = ls0 (1 + y2),
so a zero last layer gives IC(0) itself, and P_q stays symmetric positive definite.  It is
trained on solve pairs (r_k, x_k), M x_k = r_k, with the energy-norm error of one application,
    loss = (1/K) sum_k ||P_q r_k - x_k||_M^2 / ||x_k||_M^2,
the quantity conjugate gradients minimise.  Its gradient with respect to (d, lw, ls) is
written out term by term from the product rule on every power T^t (no reverse-mode
recurrence), then taken through the network by oracle/learned_factor.backward.

Plain numpy on whole vectors; vectors and blocks are (n,) or (n, K), node i = y * nx + x.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import learned_factor as lf
from . import pcg


def factor_arrays(L, nx: int):
    """(d, lw, ls) of a lower-triangular factor with the 5-point IC(0) pattern (CSR)."""
    L = sp.csr_matrix(L)
    n = L.shape[0]
    d, lw, ls = np.zeros(n), np.zeros(n), np.zeros(n)
    C = L.tocoo()
    for i, j, v in zip(C.row, C.col, C.data):
        if i == j:
            d[i] = v
        elif i - j == 1:
            lw[i] = v
        elif i - j == nx:
            ls[i] = v
        else:
            raise ValueError(f"entry ({i}, {j}) outside the 5-point IC(0) pattern")
    return d, lw, ls


def ic0_arrays(M, nx: int):
    """IC(0) of M (oracle/pcg.ic0) as (d, lw, ls)."""
    return factor_arrays(pcg.ic0(M), nx)


def _col(v):
    return v[:, None] if v.ndim == 1 else v


def n_apply(lw, ls, nx: int, V):
    """N V: (N v)_i = lw_i v_{i-1} + ls_i v_{i-nx}."""
    V = _col(V)
    out = np.zeros_like(V)
    out[1:] += lw[1:, None] * V[:-1]
    out[nx:] += ls[nx:, None] * V[:-nx]
    return out


def nt_apply(lw, ls, nx: int, V):
    """N^T V: (N^T v)_j = lw_{j+1} v_{j+1} + ls_{j+nx} v_{j+nx}."""
    V = _col(V)
    out = np.zeros_like(V)
    out[:-1] += lw[1:, None] * V[1:]
    out[:-nx] += ls[nx:, None] * V[nx:]
    return out


def t_apply(d, lw, ls, nx, V):
    """T V = -D^{-1} N V."""
    return -n_apply(lw, ls, nx, V) / d[:, None]


def tt_apply(d, lw, ls, nx, V):
    """T^T V = -N^T D^{-1} V."""
    return -nt_apply(lw, ls, nx, _col(V) / d[:, None])


def apply_B(d, lw, ls, nx: int, q: int, R):
    """B_q R = sum_{t=0}^{q} T^t D^{-1} R."""
    term = _col(R) / d[:, None]
    acc = term.copy()
    for _ in range(q):
        term = t_apply(d, lw, ls, nx, term)
        acc += term
    return acc


def apply_Bt(d, lw, ls, nx: int, q: int, Y):
    """B_q^T Y = sum_{t=0}^{q} D^{-1} (T^T)^t Y."""
    term = _col(Y).astype(np.float64, copy=True)
    acc = term.copy()
    for _ in range(q):
        term = tt_apply(d, lw, ls, nx, term)
        acc += term
    return acc / d[:, None]


def apply_P(d, lw, ls, nx: int, q: int, R):
    """P_q R = B_q^T (B_q R)."""
    return apply_Bt(d, lw, ls, nx, q, apply_B(d, lw, ls, nx, q, R))


def prec(d, lw, ls, nx: int, q: int):
    """The preconditioner as a function of one vector, for oracle/pcg.pcg."""
    return lambda r: apply_P(d, lw, ls, nx, q, r)[:, 0]


def bilinear_grad(d, lw, ls, nx: int, q: int, A_, C_):
    """Gradient of sum_k a_k^T B_q c_k (columns of A_, C_) with respect to (d, lw, ls).

    Term t of B_q is T^t D^{-1}.  With T = -D^{-1} N,
        dT = D^{-1} dD D^{-1} N - D^{-1} dN,      d(D^{-1}) = -D^{-1} dD D^{-1},
    and the product rule gives, for alpha = (T^T)^j a and beta = T^{t-1-j} D^{-1} c (0 <= j < t),
        alpha^T dT beta = sum_i alpha_i [dd_i (N beta)_i / d_i^2 - (dlw_i beta_{i-1} + dls_i beta_{i-nx}) / d_i],
    plus, from the trailing D^{-1}, -sum_i ((T^T)^t a)_i c_i dd_i / d_i^2."""
    A_, C_ = _col(A_), _col(C_)
    n = d.shape[0]
    gd, gw, gs = np.zeros(n), np.zeros(n), np.zeros(n)
    alphas = [A_.copy()]                       # (T^T)^j a, j = 0..q
    for _ in range(q):
        alphas.append(tt_apply(d, lw, ls, nx, alphas[-1]))
    betas = [C_ / d[:, None]]                  # T^u D^{-1} c, u = 0..q
    for _ in range(q):
        betas.append(t_apply(d, lw, ls, nx, betas[-1]))
    for t in range(q + 1):
        # the trailing D^{-1} of term t
        gd -= np.sum(alphas[t] * C_, axis=1) / d**2
        for j in range(t):
            al, be = alphas[j], betas[t - 1 - j]
            gd += np.sum(al * n_apply(lw, ls, nx, be), axis=1) / d**2
            bw = np.zeros_like(be)
            bw[1:] = be[:-1]
            bs = np.zeros_like(be)
            bs[nx:] = be[:-nx]
            gw -= np.sum(al * bw, axis=1) / d
            gs -= np.sum(al * bs, axis=1) / d
    return gd, gw, gs


def energy_loss(d, lw, ls, nx: int, q: int, M, R, X) -> float:
    """(1/K) sum_k ||P_q r_k - x_k||_M^2 / ||x_k||_M^2."""
    E = apply_P(d, lw, ls, nx, q, R) - _col(X)
    den = np.sum(_col(X) * (M @ _col(X)), axis=0)
    return float(np.mean(np.sum(E * (M @ E), axis=0) / den))


def energy_loss_and_grad_values(d, lw, ls, nx: int, q: int, M, R, X):
    """The loss and its gradient with respect to (d, lw, ls).

    With e_k = P r_k - x_k and g_k = 2 M e_k / (K ||x_k||_M^2), the differential of the loss is
    sum_k g_k^T dP r_k, and dP = dB^T B + B^T dB gives
    sum_k [(B r_k)^T dB g_k + (B g_k)^T dB r_k]."""
    R, X = _col(R), _col(X)
    K = R.shape[1]
    U = apply_B(d, lw, ls, nx, q, R)
    E = apply_Bt(d, lw, ls, nx, q, U) - X
    ME = M @ E
    den = np.sum(X * (M @ X), axis=0)
    loss = float(np.mean(np.sum(E * ME, axis=0) / den))
    G = 2.0 * ME / (K * den[None, :])
    Wv = apply_B(d, lw, ls, nx, q, G)
    g1 = bilinear_grad(d, lw, ls, nx, q, U, G)
    g2 = bilinear_grad(d, lw, ls, nx, q, Wv, R)
    return loss, tuple(a + b for a, b in zip(g1, g2))


def net_values(p: dict, feats: np.ndarray, d0, lw0, ls0):
    """(d, lw, ls) from the network's corrections of the IC(0) values, and its activations."""
    y, cache = lf.forward(p, feats)
    y = y.reshape(3, -1)
    return d0 * np.exp(y[0]), lw0 * (1.0 + y[1]), ls0 * (1.0 + y[2]), cache


def net_loss_and_grad(p: dict, feats: np.ndarray, d0, lw0, ls0, nx: int, q: int, M, R, X):
    """The energy loss of the network's factor and its gradient w.r.t. the parameters:
    d/dy0 = g_d d, d/dy1 = g_lw lw0, d/dy2 = g_ls ls0, then back through the convolutions."""
    d, lw, ls, cache = net_values(p, feats, d0, lw0, ls0)
    loss, (gd, gw, gs) = energy_loss_and_grad_values(d, lw, ls, nx, q, M, R, X)
    gy = np.stack([gd * d, gw * lw0, gs * ls0]).reshape(3, *feats.shape[1:])
    return loss, lf.backward(p, cache, gy)


def train(p: dict, feats, d0, lw0, ls0, nx: int, q: int, M, R, X, iters: int, lr: float,
          b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """Adam (Kingma and Ba, 2015) on the energy loss; returns the trained parameters and the
    loss before each step plus the final one."""
    p = {k: v.copy() for k, v in p.items()}
    m1 = {k: np.zeros_like(v) for k, v in p.items()}
    m2 = {k: np.zeros_like(v) for k, v in p.items()}
    losses = []
    for t in range(1, iters + 1):
        loss, g = net_loss_and_grad(p, feats, d0, lw0, ls0, nx, q, M, R, X)
        losses.append(loss)
        for k in p:
            m1[k] = b1 * m1[k] + (1 - b1) * g[k]
            m2[k] = b2 * m2[k] + (1 - b2) * g[k] ** 2
            p[k] = p[k] - lr * (m1[k] / (1 - b1**t)) / (np.sqrt(m2[k] / (1 - b2**t)) + eps)
    d, lw, ls, _ = net_values(p, feats, d0, lw0, ls0)
    losses.append(energy_loss(d, lw, ls, nx, q, M, R, X))
    return p, losses
