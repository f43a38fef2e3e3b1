"""FP64 oracle of a learned incomplete factor for the inner solves with A (an addition to the
paper, which uses direct solves; see oracle/pcg.py).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For M = -A from a 5-point stencil on a k x k grid (x fastest), the factor L keeps the IC(0)
pattern: L_ii, L_{i,i-1} (west) and L_{i,i-k} (south).  A network maps per-node features of
the operator to three corrections y = (y0, y1, y2) of the IC(0) values,

    L_ii = L0_ii exp(y0),   L_{i,i-1} = L0_{i,i-1} (1 + y1),   L_{i,i-k} = L0_{i,i-k} (1 + y2),

so a network with a zero last layer gives IC(0) itself, and the diagonal stays positive:
P = (L L^T)^{-1} is symmetric positive definite and plain CG applies.

Features (5 channels): the stencil row of M divided by its diagonal -- centre (1), west,
east, south, north (zero across the boundary).  The network is the three-layer convolution
of oracle/cnn.py with 5 input and 3 output channels.

Loss on solve pairs (r_k, x_k) with M x_k = r_k:
    loss = (1/K) sum_k ||L (L^T x_k) - r_k||^2 / ||r_k||^2,
which needs products with L and L^T only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import cnn, pcg


def stencil_features(M, k: int) -> np.ndarray:
    """(5, k, k): the stencil row of M over its diagonal (centre, west, east, south, north)."""
    M = sp.csr_matrix(M)
    n = k * k
    d = M.diagonal()
    f = np.zeros((5, n))
    f[0] = 1.0
    idx = np.arange(n)
    x, y = idx % k, idx // k
    for ch, (dx, dy) in enumerate([(-1, 0), (1, 0), (0, -1), (0, 1)], start=1):
        ok = (x + dx >= 0) & (x + dx < k) & (y + dy >= 0) & (y + dy < k)
        j = idx + dx + dy * k
        f[ch, ok] = np.asarray(M[idx[ok], j[ok]]).ravel() / d[ok]
    return f.reshape(5, k, k)


def init_params(C: int = 16, seed: int = 0, scale: float = 0.1) -> dict:
    """Weights of the 5 -> C -> C -> 3 network; the last layer starts at zero (IC(0))."""
    rng = np.random.default_rng(seed)
    return {
        "w1": rng.standard_normal((C, 5, 3, 3)) * scale / np.sqrt(5.0),
        "b1": np.zeros(C),
        "w2": rng.standard_normal((C, C, 3, 3)) * scale / np.sqrt(C),
        "b2": np.zeros(C),
        "w3": np.zeros((3, C, 3, 3)),
        "b3": np.zeros(3),
    }


def forward(p: dict, feats: np.ndarray):
    z1 = cnn.conv(feats, p["w1"], p["b1"])
    a1 = np.maximum(z1, 0.0)
    z2 = cnn.conv(a1, p["w2"], p["b2"])
    a2 = np.maximum(z2, 0.0)
    y = cnn.conv(a2, p["w3"], p["b3"])
    return y, (feats, z1, a1, z2, a2)


def backward(p: dict, cache, gy: np.ndarray) -> dict:
    feats, z1, a1, z2, a2 = cache
    g_a2, gw3, gb3 = cnn.conv_backward(a2, p["w3"], gy)
    g_z2 = g_a2 * (z2 > 0)
    g_a1, gw2, gb2 = cnn.conv_backward(a1, p["w2"], g_z2)
    g_z1 = g_a1 * (z1 > 0)
    _, gw1, gb1 = cnn.conv_backward(feats, p["w1"], g_z1)
    return {"w1": gw1, "b1": gb1, "w2": gw2, "b2": gb2, "w3": gw3, "b3": gb3}


class Pattern:
    """Positions of L0 = IC(0) of M in CSR order, and which of the three channels each is."""

    def __init__(self, M, k: int):
        self.k = k
        self.L0 = sp.csr_matrix(pcg.ic0(M))
        self.L0.sort_indices()
        n = k * k
        self.rows = np.repeat(np.arange(n), np.diff(self.L0.indptr))
        self.cols = self.L0.indices.copy()
        off = self.rows - self.cols
        self.chan = np.where(off == 0, 0, np.where(off == 1, 1, 2))
        assert np.all((off == 0) | (off == 1) | (off == k)), "5-point IC(0) pattern expected"


def factor_values(pat: Pattern, y: np.ndarray):
    """Values of L (CSR order of the pattern) from the network output y (3, k, k)."""
    yv = y.reshape(3, -1)[pat.chan, pat.rows]
    v0 = pat.L0.data
    return np.where(pat.chan == 0, v0 * np.exp(yv), v0 * (1.0 + yv))


def build_L(pat: Pattern, vals: np.ndarray) -> sp.csr_matrix:
    n = pat.k * pat.k
    return sp.csr_matrix((vals, pat.cols, pat.L0.indptr), shape=(n, n))


def loss_and_grad_values(pat: Pattern, vals: np.ndarray, R: np.ndarray, X: np.ndarray):
    """The loss over the pairs (columns of R, X) and its gradient w.r.t. the values of L."""
    L = build_L(pat, vals)
    K = R.shape[1]
    w = 1.0 / np.sum(R * R, axis=0)          # 1 / ||r_k||^2
    Y = L.T @ X
    F = L @ Y - R
    loss = float(np.sum(w * np.sum(F * F, axis=0))) / K
    Fw = F * w
    LtF = L.T @ Fw
    # d/dL_ij of sum_k w_k ||L L^T x_k - r_k||^2 = 2 sum_k w_k (F_ik Y_jk + X_ik (L^T F)_jk)
    g = 2.0 / K * (np.sum(Fw[pat.rows] * Y[pat.cols], axis=1) + np.sum(X[pat.rows] * LtF[pat.cols], axis=1))
    return loss, g


def loss_and_grad(p: dict, pat: Pattern, feats: np.ndarray, R: np.ndarray, X: np.ndarray):
    """The loss and its gradient w.r.t. the network's parameters."""
    y, cache = forward(p, feats)
    vals = factor_values(pat, y)
    loss, gv = loss_and_grad_values(pat, vals, R, X)
    # through the parametrisation: dv/dy0 = v (diagonal), dv/dy = L0 (off-diagonal)
    dv = np.where(pat.chan == 0, vals, pat.L0.data)
    gy = np.zeros((3, pat.k * pat.k))
    np.add.at(gy, (pat.chan, pat.rows), gv * dv)
    return loss, backward(p, cache, gy.reshape(3, pat.k, pat.k))
