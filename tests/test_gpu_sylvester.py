"""GPU parity of the Sylvester path A X + X B + C1 C2^T = 0 (Sec. 5.1, Alg. 4) against the FP64 oracle.

Same three levels as the Lyapunov tests:
  * the check: the GPU history at m against the oracle's Alg. 4 (with the derived
    pairing, Y~_ij = -S_ij/(lambda_i + upsilon_j)) evaluated on the GPU's own T_m and J_m,
    |d rel| <= 1e-10 max(rel, 1e-2) + 1e-13;
  * whole runs on Laplacian pairs: histories |d| <= 1e-10 + 1e-10 rel, the same m;
  * the factors: X = Z1 Z2^T against the oracle's on random probes (relative 1e-8),
    and the explicit low-rank residual of the GPU's factors.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import explicit
from oracle import sylvester as osylv

pytestmark = pytest.mark.gpu


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


def _check_on_gpu_TJ(sol, C1, C2, ms):
    s = C1.shape[1]
    bb = np.linalg.norm(C1) * np.linalg.norm(C2)
    hist = sol.history()
    worst = 0.0
    for m in ms:
        abA, gA, tA = sol.projected(m, 0)
        abB, gB, tB = sol.projected(m, 1)
        lam, Q = sla.eig_banded(abA, lower=True)
        ups, P = sla.eig_banded(abB, lower=True)
        rel = osylv.cheap_residual(lam, Q, ups, P, gA, gB, tA, tB, s) / bb
        bound = 1e-10 * max(rel, 1e-2) + 1e-13
        worst = max(worst, abs(hist[m - 1] - rel) / bound)
    return worst


def _xprobe(Z1, Z2, Z1o, Z2o, seed=0):
    u = np.random.default_rng(seed).standard_normal((Z2.shape[0], 3))
    a = Z1 @ (Z2.T @ u)
    b = Z1o @ (Z2o.T @ u)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _vc2d(k, seed, dtype=np.float64):
    kappa = np.exp(wl.gaussian_field(k, 2, seed=seed, corr_len=3.0))
    return wl.var_coeff_diffusion(kappa, dtype=dtype)


PAIRS = [  # (name, A, B, s)
    ("lap16_lap12_s2", lambda: wl.laplacian_2d(16), lambda: wl.laplacian_2d(12), 2),
    ("lap20_lap11_s1", lambda: wl.laplacian_2d(20), lambda: wl.laplacian_2d(11), 1),
    ("lap14_lap3d6_s3", lambda: wl.laplacian_2d(14), lambda: wl.laplacian_3d(6), 3),
    ("vc14_lap10_s4", lambda: _vc2d(14, 3), lambda: wl.laplacian_2d(10), 4),
]


@pytest.mark.parametrize("name,mkA,mkB,s", PAIRS, ids=[p[0] for p in PAIRS])
def test_sylvester_check_on_gpu_T(pkg, name, mkA, mkB, s):
    A, B = mkA(), mkB()
    C1 = wl.rhs(A.shape[0], s, 11)
    C2 = wl.rhs(B.shape[0], s, 12)
    sol = pkg.Solver(A, C1, B=B, C2=C2, tol=1e-9, maxit=300)
    sol.solve()
    assert sol.m >= 2
    assert _check_on_gpu_TJ(sol, C1, C2, range(1, sol.m + 1)) <= 1.0
    sol.close()


@pytest.mark.parametrize("name,mkA,mkB,s", PAIRS[:3], ids=[p[0] for p in PAIRS[:3]])
def test_sylvester_history_and_factors(pkg, name, mkA, mkB, s):
    A, B = mkA(), mkB()
    C1 = wl.rhs(A.shape[0], s, 21)
    C2 = wl.rhs(B.shape[0], s, 22)
    ref = osylv.solve(A, B, C1, C2, tol=1e-9, maxit=300)
    sol = pkg.Solver(A, C1, B=B, C2=C2, tol=1e-9, maxit=300)
    st = sol.solve()
    assert st == 0 and sol.m == ref.m
    h, ho = sol.history(), ref.history
    assert np.all(np.abs(h - ho) <= 1e-10 + 1e-10 * np.abs(ho))
    Z1, Z2 = (z.cpu().numpy() for z in sol.factor())
    Z1o, Z2o, sig = osylv.factor(A, B, C1, C2, ref)
    assert abs(Z1.shape[1] - Z1o.shape[1]) <= 1
    assert _xprobe(Z1, Z2, Z1o, Z2o) <= 1e-8
    bb = np.linalg.norm(C1) * np.linalg.norm(C2)
    rel = explicit.sylv_lowrank(A, B, Z1, Z2, C1, C2) / bb
    rel_o = explicit.sylv_lowrank(A, B, Z1o, Z2o, C1, C2) / bb
    assert abs(rel - rel_o) <= 1e-9
    sol.close()


def test_sylvester_with_B_equal_A_reproduces_lyapunov(pkg):
    """B = A, C2 = C1: Alg. 4 reduces to Prop. 3.1, so both GPU paths give the same history."""
    A = wl.laplacian_2d(18)
    C = wl.rhs(A.shape[0], 2, 5)
    ly = pkg.Solver(A, C, tol=1e-9, maxit=300)
    ly.solve()
    sy = pkg.Solver(A, C, B=A, C2=C, tol=1e-9, maxit=300)
    sy.solve()
    assert sy.m == ly.m
    h1, h2 = ly.history(), sy.history()
    assert np.all(np.abs(h1 - h2) <= 1e-12 + 1e-11 * np.abs(h1))
    Zl = ly.factor().cpu().numpy()
    Z1, Z2 = (z.cpu().numpy() for z in sy.factor())
    u = np.random.default_rng(1).standard_normal((A.shape[0], 3))
    a = Zl @ (Zl.T @ u)
    b = Z1 @ (Z2.T @ u)
    assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(a)
    ly.close()
    sy.close()


def test_sylvester_mixed_precision_fp32_operator(pkg):
    """The C3 shape at small size: A = -(3D var.-coeff. diffusion, fp32 values), B = -(2D
    Laplacian), s = 2, fp32 bulk.  The check runs in fp64 on the GPU's own T_m and J_m, so it
    matches the oracle's formula to the fp64 bound; the factors reach the tolerance in the
    explicit low-rank residual."""
    kappa = np.exp(wl.gaussian_field(10, 3, seed=1001, corr_len=1.0))
    A = wl.var_coeff_diffusion(kappa, dtype=np.float32)
    B = wl.laplacian_2d(24)
    C1 = wl.rhs(A.shape[0], 2, 3)
    C2 = wl.rhs(B.shape[0], 2, 4)
    sol = pkg.Solver(A, C1, B=B, C2=C2, tol=1e-8, maxit=400, precision="mixed", val_dtype="f32")
    st = sol.solve()
    assert st == 0
    assert _check_on_gpu_TJ(sol, C1, C2, range(1, sol.m + 1)) <= 1.0
    # the fp32 basis loses orthogonality sooner than the fp64 oracle's, which can delay the
    # first m with rel <= tol by a few steps; it never converges earlier than a tolerance allows
    ref = osylv.solve(A, B, C1, C2, tol=1e-8, maxit=400)
    assert ref.m - 2 <= sol.m <= ref.m + max(3, ref.m // 8)
    Z1, Z2 = (z.cpu().numpy().astype(np.float64) for z in sol.factor())
    rel = explicit.sylv_lowrank(A, B, Z1, Z2, C1, C2) / (np.linalg.norm(C1) * np.linalg.norm(C2))
    assert rel <= 1e-6
    sol.close()


def test_sylvester_host_outputs_equal_device_outputs(pkg):
    A, B = wl.laplacian_2d(12), wl.laplacian_2d(9)
    C1, C2 = wl.rhs(A.shape[0], 2, 1), wl.rhs(B.shape[0], 2, 2)
    a = pkg.Solver(A, C1, B=B, C2=C2, tol=1e-9, maxit=200)
    b = pkg.Solver(A, C1, B=B, C2=C2, tol=1e-9, maxit=200, inputs="host")
    a.solve()
    b.solve()
    assert np.array_equal(a.history(), b.history())
    Za1, Za2 = (z.cpu().numpy() for z in a.factor())
    Zb1, Zb2 = b.factor(out="host")
    assert np.array_equal(Za1, Zb1) and np.array_equal(Za2, Zb2)
    a.close()
    b.close()


# ---- large A, small dense B (Sec. 5.2, Alg. 5) ----
from oracle import sylvester_small as osmall  # noqa: E402

SMALLB_CASES = [  # (id, grid k, n2, s, precision, inputs)
    ("k30_n2is1_s1", 30, 1, 1, "f64", "device"),
    ("k30_n2_24_s2", 30, 24, 2, "f64", "device"),
    ("k26_n2_97_s3_host", 26, 97, 3, "f64", "host"),
    ("k33_n2_40_s4", 33, 40, 4, "f64", "device"),
    ("k30_n2_57_s2_f32x2", 30, 57, 2, "f32x2", "device"),
]


@pytest.mark.parametrize("name,k,n2,s,precision,inputs", SMALLB_CASES, ids=[c[0] for c in SMALLB_CASES])
def test_small_b_against_oracle(pkg, name, k, n2, s, precision, inputs):
    """Whole runs of the small-B path: the history of Alg. 5's residual entry by entry
    (|d| <= 1e-10 rel + 1e-14), the same m, X = Z1 Z2^T against the oracle's factors on random
    probes (relative 1e-8), and the explicit residual of the GPU's factors, dense on the host."""
    A = wl.laplacian_2d(k, shift=1.0)
    B = wl.random_snd_dense(n2, seed=n2 + 3, lam_min=0.5, lam_max=40.0)
    C1 = wl.rhs(k * k, s, seed=k + 1)
    C2 = wl.rhs(n2, s, seed=k + 2)
    tol = 1e-10
    ref = osmall.solve(A, B, C1, C2, tol=tol, maxit=300)
    sol = pkg.Solver(A, C1, B=B, C2=C2, tol=tol, maxit=300, precision=precision, trunc_eps=1e-12, inputs=inputs)
    st = sol.solve()
    assert st == 0 and ref.converged
    assert sol.m == ref.m, (sol.m, ref.m)
    h = sol.history()
    d = np.abs(h - ref.history)
    worst = float(np.max(d / (1e-10 * ref.history + 1e-14)))
    print(f"{name}: m={sol.m} max |d| {d.max():.3e} worst/bound {worst:.3f}")
    assert worst <= 1.0
    Z1, Z2 = sol.factor(out="host" if inputs == "host" else "device")
    if not isinstance(Z1, np.ndarray):
        Z1, Z2 = Z1.cpu().numpy(), Z2.cpu().numpy()
    Z1o, Z2o, _ = osmall.factor(A, C1, C2, ref, trunc_eps=1e-12)
    assert Z1.shape[1] == Z2.shape[1] and abs(Z1.shape[1] - Z1o.shape[1]) <= 1
    assert _xprobe(Z1, Z2, Z1o, Z2o) <= 1e-8
    X = Z1 @ Z2.T
    R = A @ X + X @ B + C1 @ C2.T
    rel = np.linalg.norm(R) / (np.linalg.norm(C1) * np.linalg.norm(C2))
    Xo = Z1o @ Z2o.T
    relo = np.linalg.norm(A @ Xo + Xo @ B + C1 @ C2.T) / (np.linalg.norm(C1) * np.linalg.norm(C2))
    print(f"{name}: t={Z1.shape[1]} (oracle {Z1o.shape[1]}), explicit residual {rel:.3e} (oracle {relo:.3e})")
    # truncating Y~ by trunc_eps adds at most (||A|| + ||B||) trunc_eps to the residual (eq. 2.5)
    bound = tol + (abs(A).sum(axis=1).max() + np.abs(B).sum(axis=1).max()) * 1e-12
    assert abs(rel - relo) <= 1e-3 * relo + 1e-13
    assert rel <= bound, (rel, bound)
    sol.close()


def test_small_b_check_on_gpu_T(pkg):
    """The check alone: Alg. 5 evaluated by the oracle on the GPU's own T_m (from the logged
    coefficients) against the GPU history at several m, |d rel| <= 1e-10 max(rel, 1e-2) + 1e-13."""
    k, n2, s = 28, 33, 3
    A = wl.laplacian_2d(k, shift=1.0)
    B = wl.random_snd_dense(n2, seed=5, lam_min=0.5, lam_max=40.0)
    C1, C2 = wl.rhs(k * k, s, seed=7), wl.rhs(n2, s, seed=8)
    sol = pkg.Solver(A, C1, B=B, C2=C2, tol=0.0, maxit=40)
    sol.solve()
    hist = sol.history()
    ups, P = osmall.eig_B(B)
    bb = np.linalg.norm(C1) * np.linalg.norm(C2)
    worst = 0.0
    for m in (1, 2, 7, 19, 40):
        ab, g, tn = sol.projected(m, 0)
        lam, Q = sla.eig_banded(ab, lower=True)
        rel = osmall.cheap_residual(lam, Q, ups, P, g, C2, tn, s) / bb
        worst = max(worst, abs(hist[m - 1] - rel) / (1e-10 * max(rel, 1e-2) + 1e-13))
    assert worst <= 1.0, worst
    sol.close()


def test_small_b_rejects_bad_arguments(pkg):
    from paper_1602_05033_gb300 import _lib as L

    A = wl.laplacian_2d(10, shift=1.0)
    B = wl.random_snd_dense(5, seed=1)
    C1, C2 = wl.rhs(100, 2, 1), wl.rhs(5, 2, 2)
    with pytest.raises(L.LyapError):
        pkg.Solver(A, C1, B=B, C2=C2, maxit=2)  # n2 = 5 > s maxit = 4
    bad = wl.random_snd_dense(5, seed=2)
    bad[0, 0] = np.nan
    with pytest.raises(L.LyapError):
        pkg.Solver(A, C1, B=bad, C2=C2, maxit=50)
