"""Pins of the Q1 finite-element generator (workloads.fe_mass_stiffness_2d) used by the
generalised Lyapunov oracle: facts of the discretisation, not of the method.

  * E and K = -A are symmetric positive definite.
  * The generalised eigenvalues of (K, E) are Rayleigh-Ritz values of the Laplacian on the unit
    square, so they bound the exact ones pi^2 (j^2 + l^2) from above, and bilinear elements
    converge at second order: halving h divides the error by about 4.
  * For kappa = 1 the entries of E sum to the integral of (sum of the interior basis functions)^2.
"""
import numpy as np
import scipy.linalg as sla

import workloads as wl


def _eigs(k, count=3):
    A, E = wl.fe_mass_stiffness_2d(k)
    return sla.eigh(-A.toarray(), E.toarray(), eigvals_only=True)[:count]


def test_symmetric_definite():
    A, E = wl.fe_mass_stiffness_2d(9, kappa=np.exp(wl.gaussian_field(10, 2, seed=1)))
    Ad, Ed = A.toarray(), E.toarray()
    assert np.array_equal(Ad, Ad.T) and np.array_equal(Ed, Ed.T)
    assert np.linalg.eigvalsh(Ed).min() > 0 and np.linalg.eigvalsh(-Ad).min() > 0


def test_eigenvalues_are_upper_bounds_with_second_order_error():
    exact = np.pi**2 * np.array([2.0, 5.0, 5.0])
    e7, e15 = _eigs(7) - exact, _eigs(15) - exact
    assert np.all(e7 > 0) and np.all(e15 > 0)
    ratio = e7[0] / e15[0]
    assert 3.8 < ratio < 4.2, ratio


def test_mass_matrix_integrates_the_basis():
    k = 5
    _, E = wl.fe_mass_stiffness_2d(k)
    h = 1.0 / (k + 1)
    # sum of the interior hat functions: 1 on the interior elements' shared region, and
    # on each boundary element the tensor product of the 1D sums; integrate per element with
    # the 1D Q1 mass matrices: int_0^h (a + (b - a) t/h)(c + (d - c) t/h) dt = h (2ac + ad + bc + 2bd)/6
    def m1(a, b, c, d):
        return h * (2 * a * c + a * d + b * c + 2 * b * d) / 6.0
    total = 0.0
    for ey in range(k + 1):
        for ex in range(k + 1):
            # 1D values of the summed interior hats at the element's two nodes, per direction
            vx = (0.0 if ex == 0 else 1.0, 0.0 if ex == k else 1.0)
            vy = (0.0 if ey == 0 else 1.0, 0.0 if ey == k else 1.0)
            total += m1(*vx, *vx) * m1(*vy, *vy)
    assert abs(E.sum() - total) <= 1e-13 * total
