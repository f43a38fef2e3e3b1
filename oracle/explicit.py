"""Explicit residual norms of a low-rank approximate solution (pins, not the method).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For X ~= Z Z^T the Lyapunov residual R = A Z Z^T + Z Z^T A + C C^T equals
U M U^T with U = [A Z, Z, C] and M = [[0, I, 0], [I, 0, 0], [0, 0, I]].  With a
thin QR U = Q_U R_U, ||R||_F = ||R_U M R_U^T||_F exactly, in O(n (2t+s)^2)
operations; the dense form is used only for small n.
"""
from __future__ import annotations

import numpy as np


def lyap_dense(A, Z, C):
    A = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    X = Z @ Z.T
    R = A @ X + X @ A + C @ C.T
    return float(np.linalg.norm(R, "fro"))


def lyap_lowrank(A, Z, C):
    t, s = Z.shape[1], C.shape[1]
    U = np.hstack([A @ Z, Z, C])
    _, RU = np.linalg.qr(U, mode="reduced")
    Mm = np.zeros((2 * t + s, 2 * t + s))
    Mm[:t, t:2 * t] = np.eye(t)
    Mm[t:2 * t, :t] = np.eye(t)
    Mm[2 * t:, 2 * t:] = np.eye(s)
    return float(np.linalg.norm(RU @ Mm @ RU.T, "fro"))


def sylv_dense(A, B, Z1, Z2, C1, C2):
    A = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    B = B.toarray() if hasattr(B, "toarray") else np.asarray(B)
    X = Z1 @ Z2.T
    return float(np.linalg.norm(A @ X + X @ B + C1 @ C2.T, "fro"))


def sylv_lowrank(A, B, Z1, Z2, C1, C2):
    """R = [A Z1, Z1, C1] [Z2, B Z2, C2]^T; ||R||_F = ||R1 R2^T||_F from two thin QRs."""
    U1 = np.hstack([A @ Z1, Z1, C1])
    U2 = np.hstack([Z2, B @ Z2, C2])
    _, R1 = np.linalg.qr(U1, mode="reduced")
    _, R2 = np.linalg.qr(U2, mode="reduced")
    return float(np.linalg.norm(R1 @ R2.T, "fro"))
