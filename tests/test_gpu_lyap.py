"""GPU parity of the Lyapunov path (through the C ABI) against the FP64 oracle.

Three levels, each with its own tolerance:
  * the convergence check itself: the history the GPU records at m is compared
    with the oracle's Prop. 3.1 evaluated on the GPU's own T_m, gamma and
    tau_{m+1,m} (exported by lyap_projected_matrix), at every m.  Both evaluate
    the same function of the same fp64 data, so
        |rel_gpu(m) - rel_oracle(T_gpu)(m)| <= 1e-10 rel + HIST_ATOL.
  * the block Lanczos recurrence: T_m from the GPU (projections and Cholesky QR from one reduction) against
    T_m from the oracle (textbook MGS + Householder QR) while local
    orthogonality keeps them close: |dT| <= 1e-11 ||T||.
  * the whole run: the residual histories and iteration counts of the two
    independent implementations, |d rel| <= HIST_ATOL + HIST_RTOL * rel, on
    operators where finite-precision Lanczos stays reproducible (the Laplacians);
    the factor X = Z Z^T is compared on random vectors, relative 1e-8.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import explicit
from oracle import lyap as olyap

pytestmark = pytest.mark.gpu

# relative 1e-10 per entry, plus an absolute floor (in units of beta^2) for entries whose
# rounding is absolute: the last rows of eigenvectors of converged Ritz values are computed to
# absolute, not relative, accuracy, so late entries carry an absolute error of a few eps
HIST_RTOL = 1e-10
HIST_ATOL = 1e-14


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


def _hist_ok(h_gpu, h_ref):
    n = min(len(h_gpu), len(h_ref))
    d = np.abs(h_gpu[:n] - h_ref[:n])
    bound = HIST_ATOL + HIST_RTOL * np.abs(h_ref[:n])
    return bool(np.all(d <= bound)), float(np.max(d / bound)) if n else 0.0


def _xprobe(Z, Zo, seed=0):
    u = np.random.default_rng(seed).standard_normal((Z.shape[0], 4))
    a = Z @ (Z.T @ u)
    b = Zo @ (Zo.T @ u)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _solve_both(pkg, A, C, tol, maxit, **kw):
    ref = olyap.solve(A, C, tol=tol, maxit=maxit)
    sol = pkg.Solver(A, C, tol=tol, maxit=maxit, **kw)
    st = sol.solve()
    return ref, sol, st


def _check_on_gpu_T(sol, C, ms):
    """max over m of |GPU history - oracle Prop. 3.1 on the GPU's T_m| / bound."""
    s = C.shape[1]
    beta2 = np.linalg.norm(C) ** 2
    hist = sol.history()
    worst = 0.0
    for m in ms:
        ab, gam, tau = sol.projected(m)
        lam, Q = sla.eig_banded(ab, lower=True)
        rel = olyap.cheap_residual(lam, Q, gam, tau, s) / beta2
        bound = HIST_RTOL * rel + HIST_ATOL
        worst = max(worst, abs(hist[m - 1] - rel) / bound)
    return worst


CASES = [  # (name, operator builder, s, tol, maxit)
    ("lap2d20_s2", lambda: wl.laplacian_2d(20), 2, 1e-9, 400),
    ("lap2d14_s3", lambda: wl.laplacian_2d(14), 3, 1e-9, 400),
    ("lap2d16_s4", lambda: wl.laplacian_2d(16), 4, 1e-9, 400),
    ("lap2d33_s4", lambda: wl.laplacian_2d(33), 4, 1e-9, 400),
    ("lap3d12_s4", lambda: wl.laplacian_3d(12), 4, 1e-9, 400),
]


@pytest.mark.parametrize("name,make,s,tol,maxit", CASES, ids=[c[0] for c in CASES])
def test_check_matches_oracle_formula_on_gpu_T(pkg, name, make, s, tol, maxit):
    A = make()
    C = wl.rhs(A.shape[0], s, 7)
    sol = pkg.Solver(A, C, tol=tol, maxit=maxit)
    sol.solve()
    assert _check_on_gpu_T(sol, C, range(1, sol.m + 1)) <= 1.0
    sol.close()


def test_dense_spectrum_operator(pkg):
    """A dense SND matrix stored as CSR (every row has n entries: wide SELL slices).
    Its extreme Ritz values converge within a few steps, after which the two
    implementations' Lanczos runs drift apart in finite precision; the check is
    compared on the GPU's own T_m at every m, and T_m itself while the runs agree."""
    import scipy.sparse as sp

    A = sp.csr_matrix(wl.random_snd_dense(300, seed=5, lam_min=1.0, lam_max=500.0))
    C = wl.rhs(300, 3, 6)
    ref, sol, st = _solve_both(pkg, A, C, 1e-10, 40)
    assert _check_on_gpu_T(sol, C, range(1, sol.m + 1)) <= 1.0
    for m in (1, 2, 4, 6):
        ab, _, _ = sol.projected(m)
        abo = olyap.band_T(ref.log, m)
        assert np.max(np.abs(ab - abo)) <= 1e-11 * np.max(np.abs(abo)), m
    sol.close()


@pytest.mark.parametrize("s,k,seed", [(1, 30, 1), (2, 20, 1), (3, 14, 2), (4, 16, 3)])
def test_projected_matrix_matches_oracle(pkg, s, k, seed):
    A = wl.laplacian_2d(k)
    C = wl.rhs(A.shape[0], s, seed)
    ref = olyap.solve(A, C, tol=0.0, maxit=12)
    sol = pkg.Solver(A, C, tol=0.0, maxit=12)
    sol.solve()
    for m in (1, 5, 12):
        ab, gam, tau = sol.projected(m)
        abo = olyap.band_T(ref.log, m)
        scale = np.max(np.abs(abo))
        assert np.max(np.abs(ab - abo)) <= 1e-11 * scale
        assert np.max(np.abs(tau - ref.log.tau_next[m - 1])) <= 1e-11 * scale
    assert np.max(np.abs(gam - ref.log.gamma)) <= 1e-13 * np.max(np.abs(ref.log.gamma))
    sol.close()


def test_config_c1_history_and_factor(pkg):
    """Lyapunov, 2D Laplacian 50x50, s = 1, tol 1e-8 (the small fp64 workload)."""
    P = wl.config_c1(0)
    ref, sol, st = _solve_both(pkg, P.A, P.C1, P.tol, P.maxit)
    assert st == 0 and sol.m == ref.m
    ok, worst = _hist_ok(sol.history(), ref.history)
    assert ok, worst
    Z = sol.factor().cpu().numpy()
    Zo, _ = olyap.factor(P.A, P.C1, ref)
    assert abs(Z.shape[1] - Zo.shape[1]) <= 1
    assert _xprobe(Z, Zo) <= 1e-8
    rel = explicit.lyap_lowrank(P.A, Z, P.C1) / ref.log.beta**2
    rel_o = explicit.lyap_lowrank(P.A, Zo, P.C1) / ref.log.beta**2
    assert abs(rel - rel_o) <= 1e-9
    sol.close()


@pytest.mark.parametrize("s,k,seed", [(2, 20, 1), (3, 14, 2), (4, 16, 3), (4, 33, 4)])
def test_block_sizes_laplacian(pkg, s, k, seed):
    A = wl.laplacian_2d(k)
    C = wl.rhs(A.shape[0], s, seed)
    ref, sol, st = _solve_both(pkg, A, C, 1e-9, 400)
    assert st == 0 and sol.m == ref.m
    ok, worst = _hist_ok(sol.history(), ref.history)
    assert ok, worst
    Z = sol.factor().cpu().numpy()
    Zo, _ = olyap.factor(A, C, ref)
    assert _xprobe(Z, Zo) <= 1e-8
    sol.close()


def test_host_inputs_match_device_inputs(pkg):
    A = wl.laplacian_2d(18)
    C = wl.rhs(A.shape[0], 2, 9)
    a = pkg.Solver(A, C, tol=1e-9, maxit=300, inputs="device")
    b = pkg.Solver(A, C, tol=1e-9, maxit=300, inputs="host")
    a.solve()
    b.solve()
    assert a.m == b.m
    assert np.array_equal(a.history(), b.history())  # same kernels, same bits
    Za = a.factor().cpu().numpy()
    Zb = b.factor(out="host")
    assert np.array_equal(Za, Zb)
    a.close()
    b.close()


def test_check_period(pkg):
    """check_every = d tests only m = d, 2d, ... (the paper's periodic check)."""
    A = wl.laplacian_2d(20)
    C = wl.rhs(A.shape[0], 1, 2)
    ref = olyap.solve(A, C, tol=1e-8, maxit=500, check_every=5)
    sol = pkg.Solver(A, C, tol=1e-8, maxit=500, check_every=5)
    sol.solve()
    assert sol.m == ref.m and sol.m % 5 == 0
    h = sol.history()
    assert np.all(np.isnan(h[np.arange(len(h)) % 5 != 4]))
    ok, worst = _hist_ok(h[4::5], ref.history[4::5])
    assert ok, worst


def test_not_converged_within_maxit(pkg):
    from paper_1602_05033_gb300 import _lib

    A = wl.laplacian_2d(30)
    C = wl.rhs(A.shape[0], 1, 3)
    sol = pkg.Solver(A, C, tol=1e-12, maxit=20)
    assert sol.solve() == _lib.LYAP_NOT_CONVERGED
    assert sol.m == 20 and len(sol.history()) == 20
    ref = olyap.solve(A, C, tol=1e-12, maxit=20)
    ok, worst = _hist_ok(sol.history(), ref.history)
    assert ok, worst


def test_nonfinite_rhs_rejected(pkg):
    from paper_1602_05033_gb300 import _lib

    A = wl.laplacian_2d(10)
    C = wl.rhs(100, 2, 1)
    C[7, 1] = np.nan
    sol = pkg.Solver(A, C, tol=1e-8, maxit=50)
    with pytest.raises(_lib.LyapError) as e:
        sol.solve()
    assert e.value.status == _lib.LYAP_ERR_NONFINITE


def test_rank_deficient_rhs_is_breakdown(pkg):
    from paper_1602_05033_gb300 import _lib

    A = wl.laplacian_2d(10)
    C = wl.rhs(100, 2, 1)
    C[:, 1] = C[:, 0]
    sol = pkg.Solver(A, C, tol=1e-8, maxit=50)
    with pytest.raises(_lib.LyapError) as e:
        sol.solve()
    assert e.value.status == _lib.LYAP_ERR_BREAKDOWN


def test_indefinite_operator_detected(pkg):
    from paper_1602_05033_gb300 import _lib

    A = wl.laplacian_2d(10, shift=-2.0 * 8 * 11**2)  # shifted to positive definite
    C = wl.rhs(100, 1, 1)
    sol = pkg.Solver(A, C, tol=1e-8, maxit=30)
    with pytest.raises(_lib.LyapError) as e:
        sol.solve()
    assert e.value.status == _lib.LYAP_ERR_NOT_NEGDEF


def test_speculative_chunks_follow_the_residual_trend(pkg):
    """The chunk of steps launched ahead of its checks is sized from the residual trend (the
    convergence test is unchanged): the result equals the oracle's m and history, and the steps
    run past the converged m stay below what a blindly doubled chunk can leave (up to 63: the
    rest of the converging chunk of up to 32, plus a whole speculative chunk of 32)."""
    A = wl.laplacian_3d(14)
    C = wl.rhs(A.shape[0], 4, 21)
    ref, sol, st = _solve_both(pkg, A, C, 1e-9, 400)
    assert st == 0 and sol.m == ref.m
    ok, worst = _hist_ok(sol.history(), ref.history)
    assert ok, worst
    ph = sol.phase_times()
    wasted, late_checks = ph[7], ph[8]
    print(f"m={sol.m}: steps past m {wasted:.0f}, checks past m {late_checks:.0f}")
    assert 0 <= late_checks <= wasted < 48
    sol.close()


ADAPTIVE_TARGETS = [11, 13, 19, 27, 37, 53, 71]


def test_adaptive_schedule_finds_the_first_converged_m(pkg):
    """The adaptive check schedule (every m up to 8, every 8th m until the residual trend
    predicts tol within reach, then every m; the m skipped before the first converged check are
    checked afterwards).  For each target m0 the tolerance is placed between the oracle's
    residuals at m0 - 1 and m0 on a stretch where the history decreases, so the first m meeting
    it is m0: the GPU must return exactly m0, its checked entries must match the oracle's
    history, and the skipped entries are NaN.  Targets inside the sparse stretch take the
    backfill path."""
    A = wl.laplacian_2d(40)
    C = wl.rhs(A.shape[0], 2, 5)
    full = olyap.solve(A, C, tol=0.0, maxit=90).history
    skipped_total = 0
    for m0 in ADAPTIVE_TARGETS:
        assert np.all(np.diff(full[: m0]) < 0), m0
        tol = float(np.sqrt(full[m0 - 2] * full[m0 - 1]))
        sol = pkg.Solver(A, C, tol=tol, maxit=200, check_every="adaptive")
        st = sol.solve()
        assert st == 0 and sol.m == m0, (m0, sol.m)
        h = sol.history()
        chk = ~np.isnan(h)
        assert chk[: min(8, m0)].all() and chk[m0 - 1]
        ok, worst = _hist_ok(h[chk], full[: m0][chk])
        assert ok, (m0, worst)
        ph = sol.phase_times()
        skipped_total += int((~chk).sum())
        print(f"m0={m0}: checks {ph[9]:.0f} (past m {ph[8]:.0f}), skipped {int((~chk).sum())}, worst/bound {worst:.3f}")
        sol.close()
    assert skipped_total > 0


@pytest.mark.parametrize("s,k,tol", [(1, 50, 1e-8), (4, 14, 1e-9), (3, 24, 1e-10)])
def test_adaptive_schedule_matches_oracle_run(pkg, s, k, tol):
    """Whole runs under the adaptive schedule: the same m as the oracle checking every m, the
    checked entries within the history bound, the factor's X on probes within 1e-8."""
    A = wl.laplacian_3d(k) if s == 4 else wl.laplacian_2d(k)
    C = wl.rhs(A.shape[0], s, 31 + s)
    ref = olyap.solve(A, C, tol=tol, maxit=600)
    sol = pkg.Solver(A, C, tol=tol, maxit=600, check_every="adaptive")
    st = sol.solve()
    assert st == 0 and sol.m == ref.m, (sol.m, ref.m)
    h = sol.history()
    chk = ~np.isnan(h)
    ok, worst = _hist_ok(h[chk], ref.history[chk])
    assert ok, worst
    ph = sol.phase_times()
    print(f"s={s} k={k}: m={sol.m}, checks {ph[9]:.0f} of {sol.m}, worst/bound {worst:.3f}")
    assert ph[9] < sol.m + ph[8]
    Z = sol.factor().cpu().numpy()
    Zo, _ = olyap.factor(A, C, ref)
    assert _xprobe(Z, Zo) <= 1e-8
    sol.close()
