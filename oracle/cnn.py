"""FP64 oracle of 3x3 convolution layers (zero padding) and their backward passes, which the
inner-solve networks of the extended Krylov method are built from (oracle/learned_factor.py,
oracle/neumann_ic.py).  The three-layer network here (1 -> C -> C -> 1 channels, ReLU after the
first two, applied to a residual laid out on the operator's grid) and its least-squares and
energy-norm losses are the first design of that preconditioner, a correction to Jacobi scaling,
kept with their pins; the GPU path now learns corrections of the IC(0) factor values instead.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy loops over the nine taps;
parameters are a dict with w1 (C,1,3,3), b1 (C), w2 (C,C,3,3), b2 (C), w3 (1,C,3,3), b3 (1).
Images are (channels, ny, nx) with x fastest, so a grid vector u of length ny*nx is the image
u.reshape(ny, nx).  Tap (dy, dx) of a filter multiplies the input at (y + dy - 1, x + dx - 1).
"""
from __future__ import annotations

import numpy as np


def init_params(C: int = 16, seed: int = 0, scale: float = 0.1) -> dict:
    rng = np.random.default_rng(seed)
    return {
        "w1": rng.standard_normal((C, 1, 3, 3)) * scale,
        "b1": rng.standard_normal(C) * 0.01,
        "w2": rng.standard_normal((C, C, 3, 3)) * scale / np.sqrt(C),
        "b2": rng.standard_normal(C) * 0.01,
        "w3": rng.standard_normal((1, C, 3, 3)) * scale / np.sqrt(C),
        "b3": np.zeros(1),
    }


def _shift(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """out[..., y, x] = x[..., y + dy - 1, x + dx - 1] (zero outside)."""
    out = np.zeros_like(x)
    ny, nx = x.shape[-2:]
    oy, ox = dy - 1, dx - 1
    ys = slice(max(0, -oy), min(ny, ny - oy))
    xs = slice(max(0, -ox), min(nx, nx - ox))
    yi = slice(max(0, oy), min(ny, ny + oy))
    xi = slice(max(0, ox), min(nx, nx + ox))
    out[..., ys, xs] = x[..., yi, xi]
    return out


def conv(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[co] = b[co] + sum_ci sum_taps w[co, ci, dy, dx] x[ci](y + dy - 1, x + dx - 1)."""
    y = np.zeros((w.shape[0],) + x.shape[1:])
    for dy in range(3):
        for dx in range(3):
            xs = _shift(x, dy, dx)
            y += np.einsum("oc,cyx->oyx", w[:, :, dy, dx], xs)
    return y + b[:, None, None]


def conv_backward(x: np.ndarray, w: np.ndarray, gy: np.ndarray):
    """Gradients of sum(gy * conv(x, w, b)) with respect to x, w and b."""
    gw = np.zeros_like(w)
    gx = np.zeros_like(x)
    for dy in range(3):
        for dx in range(3):
            xs = _shift(x, dy, dx)
            gw[:, :, dy, dx] = np.einsum("oyx,cyx->oc", gy, xs)
            # the input at (y + dy - 1, x + dx - 1) received w * gy(y, x): shift gy the other way
            gx += _shift(np.einsum("oc,oyx->cyx", w[:, :, dy, dx], gy), 2 - dy, 2 - dx)
    gb = gy.sum(axis=(1, 2))
    return gx, gw, gb


def forward(p: dict, u: np.ndarray, shape):
    """CNN(u) for a grid vector u (length ny*nx); returns the output vector and the activations."""
    ny, nx = shape
    x0 = u.reshape(1, ny, nx)
    z1 = conv(x0, p["w1"], p["b1"])
    a1 = np.maximum(z1, 0.0)
    z2 = conv(a1, p["w2"], p["b2"])
    a2 = np.maximum(z2, 0.0)
    y = conv(a2, p["w3"], p["b3"])
    return y.reshape(-1), (x0, z1, a1, z2, a2)


def backward(p: dict, cache, gy_vec: np.ndarray, shape) -> dict:
    """Gradients of sum(gy * CNN(u)) with respect to the parameters."""
    ny, nx = shape
    x0, z1, a1, z2, a2 = cache
    gy = gy_vec.reshape(1, ny, nx)
    g_a2, gw3, gb3 = conv_backward(a2, p["w3"], gy)
    g_z2 = g_a2 * (z2 > 0)
    g_a1, gw2, gb2 = conv_backward(a1, p["w2"], g_z2)
    g_z1 = g_a1 * (z1 > 0)
    _, gw1, gb1 = conv_backward(x0, p["w1"], g_z1)
    return {"w1": gw1, "b1": gb1, "w2": gw2, "b2": gb2, "w3": gw3, "b3": gb3}


def loss_and_grad(p: dict, R: np.ndarray, X: np.ndarray, shape):
    """L = (1/K) sum_k ||CNN(r_k) - x_k||^2 over training pairs (columns of R and X, each pair
    scaled so that ||r_k|| = 1) and its gradient."""
    K = R.shape[1]
    L = 0.0
    g = {k: np.zeros_like(v) for k, v in p.items()}
    for k in range(K):
        nr = np.linalg.norm(R[:, k])
        r, x = R[:, k] / nr, X[:, k] / nr
        y, cache = forward(p, r, shape)
        d = y - x
        L += float(d @ d) / K
        gk = backward(p, cache, 2.0 * d / K, shape)
        for key in g:
            g[key] += gk[key]
    return L, g


def energy_loss_and_grad(p: dict, A, R: np.ndarray, X: np.ndarray, shape, jacobi: bool = False):
    """L = (1/K) sum_k ||y_k - x_k||^2_{-A} / ||x_k||^2_{-A} over solve pairs A x_k = r_k
    (A symmetric negative definite, so -A defines the energy norm conjugate gradients minimise),
    each pair scaled to ||r_k|| = 1, and its gradient; y_k = CNN(r_k), or with ``jacobi``
    y_k = r_k / diag(A) + CNN(r_k) (the network as a correction to Jacobi scaling).  d/dy of the
    k-th term is 2 (-A)(y - x) / ||x||^2_{-A} = 2 (r - A y) / ||x||^2_{-A}."""
    K = R.shape[1]
    L = 0.0
    g = {k: np.zeros_like(v) for k, v in p.items()}
    dA = A.diagonal()
    for k in range(K):
        nr = np.linalg.norm(R[:, k])
        r, x = R[:, k] / nr, X[:, k] / nr
        y, cache = forward(p, r, shape)
        if jacobi:
            y = y + r / dA
        d = y - x
        ex = float(x @ (-(A @ x)))
        L += float(d @ (-(A @ d))) / ex / K
        gk = backward(p, cache, 2.0 * (r - A @ y) / ex / K, shape)
        for key in g:
            g[key] += gk[key]
    return L, g
