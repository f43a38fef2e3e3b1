"""GPU parity of the generalised Lyapunov path A X E + E X A + C C^T = 0 (E symmetric positive
definite, the mass-matrix example of Sec. 6) against the FP64 oracle, which forms the Cholesky
factor E = L L^T and runs the standard method on L^{-1} A L^{-T} (dense, small n), with the
block Gram-Schmidt against every stored block as the GPU does (on these operators the plain
recurrence loses orthogonality within a few tens of steps).

The GPU never forms L: it runs block Lanczos with an E-orthonormal basis and conjugate-gradient
solves with E (to relative residual 1e-13), so its T_m agrees with the oracle's up to the inner
solves' accuracy.  Checked per case:
  * the same m, and the history entry by entry within 1e-9 relative + 1e-13 (the inner solves
    add a relative perturbation of about 1e-13 to every coefficient, amplified by the check);
  * X = Z Z^T against the oracle's factor on random probes (relative 1e-8);
  * the explicit residual ||A X E + E X A + C C^T||_F of the GPU's factor, dense on the host, no
    more than twice the oracle's plus the truncation allowance.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import lyap_general as lg

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-9, 1e-13


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1602_05033_gb300 as p
    from paper_1602_05033_gb300 import _lib
    from paper_1602_05033_gb300 import build as b

    b.build()
    _lib.load()
    return p


# s = 1 only with variable coefficients: the constant-coefficient square grid has double
# eigenvalues, which a single starting vector sees as one direction until rounding splits them;
# the oracle's own history then moves by tens of percent late in the run under a 1e-14
# perturbation of the operator, so no implementation can match it there
CASES = [("fe18_s1_kappa", 18, 1, 0.5), ("fe15_s2", 15, 2, None), ("fe18_s4", 18, 4, None), ("fe16_s2_kappa", 16, 2, 1.0)]


@pytest.mark.parametrize("name,k,s,sig", CASES, ids=[c[0] for c in CASES])
def test_generalized_against_oracle(pkg, name, k, s, sig):
    kappa = None if sig is None else np.exp(sig * wl.gaussian_field(k + 1, 2, seed=k, corr_len=3.0))
    A, E = wl.fe_mass_stiffness_2d(k, kappa)
    C = wl.rhs(k * k, s, seed=k + s)
    tol = 1e-10
    ref = lg.solve(A, E, C, tol=tol, maxit=300)
    assert ref.inner.converged
    g = pkg.Generalized(A, E, C, tol=tol, maxit=300)
    st = g.solve()
    assert st == 0 and g.m == ref.inner.m, (g.m, ref.inner.m)
    h = g.history()
    d = np.abs(h - ref.inner.history)
    worst = float(np.max(d / (RTOL * ref.inner.history + ATOL)))
    stats = g.stats()
    print(f"{name}: m={g.m} max |d| {d.max():.3e} max rel {np.max(d / ref.inner.history):.3e} worst/bound "
          f"{worst:.3f}; E-solves {stats['e_solves']}, CG iterations {stats['cg_iterations']} (max {stats['cg_max']})")
    assert worst <= 1.0
    Z = g.factor().cpu().numpy()
    Zo, _ = lg.factor(ref)
    u = np.random.default_rng(1).standard_normal((Z.shape[0], 3))
    px = np.linalg.norm(Z @ (Z.T @ u) - Zo @ (Zo.T @ u)) / np.linalg.norm(Zo @ (Zo.T @ u))
    assert px <= 1e-8, px
    Ad, Ed = A.toarray(), E.toarray()

    def expl(Zf):
        X = Zf @ Zf.T
        return np.linalg.norm(Ad @ X @ Ed + Ed @ X @ Ad + C @ C.T)

    r, ro = expl(Z), expl(Zo)
    print(f"{name}: t={Z.shape[1]} (oracle {Zo.shape[1]}), explicit residual {r:.3e} (oracle {ro:.3e})")
    assert r <= 2 * ro + 1e-12 * np.linalg.norm(C) ** 2
    g.close()


def test_identity_mass_matrix_is_the_standard_equation(pkg):
    """E = I: the equation is the standard one; the generalised path matches the oracle's
    standard-equation history (full reorthogonalisation) and the CG solves with I take one
    iteration each."""
    import scipy.sparse as sp

    A = wl.laplacian_2d(14)
    C = wl.rhs(A.shape[0], 2, seed=9)
    I = sp.identity(A.shape[0], format="csr")
    ref = lg.solve(A, I, C, tol=1e-9, maxit=300)
    g = pkg.Generalized(A, I, C, tol=1e-9, maxit=300)
    assert g.solve() == 0 and g.m == ref.inner.m
    h = g.history()
    assert np.all(np.abs(h - ref.inner.history) <= 1e-13 + 1e-10 * ref.inner.history)
    assert g.stats()["cg_max"] <= 8  # one iteration solves; convergence is read every 8 iterations
    g.close()
