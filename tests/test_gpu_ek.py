"""GPU parity of the extended Krylov path (Sec. 4) and of its inner-solve preconditioners.

  * EK with conjugate-gradient inner solves (inner tolerance 1e-13; Jacobi or IC(0)) against the
    FP64 oracle with exact solves: the same iteration count and histories within 1e-9 rel.
    (+1e-12), the factor by X probes;
  * the IC(0) factor values from the anti-diagonal sweep against oracle/pcg.ic0 (square, ragged and
    1024-wide grids), and the truncated-Neumann application P R against oracle/neumann_ic;
  * the network's values, energy loss and gradient (bf16 weights and activations, fp32
    accumulation, the 16 -> 16 layer on the tensor cores) against the fp64 oracle evaluated with
    the same bf16-rounded weights;
  * the gain: the network trained on the method's first solve pair takes fewer inner CG iterations
    than IC(0) with the same application, with the same EK result.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as wl
from oracle import ek as oek
from oracle import learned_factor as lf
from oracle import neumann_ic as ni

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


def _vc2d(k, seed, sigma=1.5, corr=4.0):
    kappa = np.exp(sigma * wl.gaussian_field(k, 2, seed=seed, corr_len=corr))
    return wl.var_coeff_diffusion(kappa)


def _scaled_lap(nx, ny, seed):
    """D (-(I (x) T_nx + T_ny (x) I)) D with a random positive diagonal D: a 5-point operator on a
    non-square nx x ny grid (x fastest), symmetric negative definite."""
    def t(m):
        return sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    L = sp.kron(sp.identity(ny), t(nx)) + sp.kron(t(ny), sp.identity(nx))
    D = sp.diags(np.exp(0.5 * np.random.default_rng(seed).standard_normal(nx * ny)))
    return sp.csr_matrix(-(D @ L @ D))


def _xprobe(Z, Zo, seed=0):
    u = np.random.default_rng(seed).standard_normal((Z.shape[0], 3))
    a = Z @ (Z.T @ u)
    b = Zo @ (Zo.T @ u)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name,mk,s,grid,prec", [("lap2d20_s1", lambda: wl.laplacian_2d(20), 1, None, "jacobi"),
                                                 ("vc2d16_s2", lambda: _vc2d(16, 3), 2, None, "jacobi"),
                                                 ("vc2d16_s2_ic0", lambda: _vc2d(16, 3), 2, (16, 16), "ic0"),
                                                 ("lap2d12_s4_ic0", lambda: wl.laplacian_2d(12), 4, (12, 12), "ic0")])
def test_ek_matches_oracle(pkg, name, mk, s, grid, prec):
    A = mk()
    C = wl.rhs(A.shape[0], s, 9)
    ref = oek.solve(A, C, tol=1e-9, maxit=40)
    e = pkg.ExtendedKrylov(A, C, tol=1e-9, maxit=40, inner_tol=1e-13, grid=grid)
    st = e.solve(prec)
    assert st == 0 and e.m == ref.m
    h = e.history()
    assert np.all(np.abs(h - ref.history) <= 1e-12 + 1e-9 * np.abs(ref.history)), np.max(np.abs(h - ref.history))
    Z = e.factor().cpu().numpy()
    Zo, _ = oek.factor(ref)
    assert _xprobe(Z, Zo) <= 1e-7
    e.close()


def _M(A):
    return sp.csr_matrix(-A)


@pytest.mark.parametrize("nx,ny", [(16, 16), (13, 9), (1024, 3)])
def test_ic0_values_and_application_match_oracle(pkg, nx, ny):
    A = _scaled_lap(nx, ny, 5) if nx != ny else _vc2d(nx, 5)
    n = A.shape[0]
    e = pkg.ExtendedKrylov(A, np.ones((n, 1)), maxit=2, grid=(nx, ny))
    assert e.precond_status() == 0
    d, lw, ls = e.precond_values("ic0")
    d0, lw0, ls0 = ni.ic0_arrays(_M(A), nx)
    for got, ref in ((d, d0), (lw, lw0), (ls, ls0)):
        assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    R = np.random.default_rng(1).standard_normal((n, 3))
    Z = e.precond_apply("ic0", R)
    Zo = ni.apply_P(d0, lw0, ls0, nx, 3, R)
    assert np.allclose(Z, Zo, rtol=1e-12, atol=1e-12 * np.abs(Zo).max())
    e.close()


def test_precondition_status_rejects_a_non_grid_operator(pkg):
    A = sp.csr_matrix(wl.laplacian_2d(8))
    A = A + sp.csr_matrix(([-1.0, -1.0], ([0, 63], [63, 0])), shape=A.shape)  # a coupling outside the stencil
    e = pkg.ExtendedKrylov(A.tocsr(), np.ones((64, 1)), maxit=2, grid=(8, 8))
    assert e.precond_status() & 1
    from paper_1602_05033_gb300 import _lib

    with pytest.raises(_lib.LyapError):
        e.solve("ic0")
    e.close()


def _flat(p):
    return np.concatenate([p["w1"].ravel(), p["b1"], p["w2"].ravel(), p["b2"], p["w3"].ravel(), p["b3"]]).astype(np.float32)


def _unflat(v, C=16):
    k = 0
    out = {}
    for key, shape in (("w1", (C, 5, 3, 3)), ("b1", (C,)), ("w2", (C, C, 3, 3)), ("b2", (C,)), ("w3", (3, C, 3, 3)),
                       ("b3", (3,))):
        sz = int(np.prod(shape))
        out[key] = np.asarray(v[k:k + sz], dtype=np.float64).reshape(shape)
        k += sz
    return out


def _bf16(v):
    """Round float32 values to bfloat16 (round to nearest even), back to float64."""
    u = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _params(seed, scale=0.3, w3=0.05):
    rng = np.random.default_rng(seed)
    p = lf.init_params(16, seed, scale)
    p["b1"] = rng.standard_normal(16) * 0.05
    p["b2"] = rng.standard_normal(16) * 0.05
    p["w3"] = rng.standard_normal(p["w3"].shape) * w3
    p["b3"] = rng.standard_normal(3) * 0.01
    flat = _flat(p)
    pq = _unflat(_bf16(flat))
    for key in ("b1", "b2", "b3"):
        pq[key] = _unflat(flat)[key]  # biases stay fp32
    return flat, pq


@pytest.mark.parametrize("k", [12, 21])
def test_network_values_and_gradient_match_oracle(pkg, k):
    A = _vc2d(k, 7, corr=3.0)
    n = A.shape[0]
    M = _M(A)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((n, 2))
    B = A @ X
    flat, pq = _params(4)
    e = pkg.ExtendedKrylov(A, rng.standard_normal((n, 1)), maxit=4, grid=(k, k))
    d0, lw0, ls0 = ni.ic0_arrays(M, k)
    feats = lf.stencil_features(M, k)
    # the values: corrections y of the IC(0) values, fp64 oracle with the bf16 weights
    R = rng.standard_normal((n, 2))
    Z = e.precond_apply("learned", R, params=flat)
    d, lw, ls = e.precond_values("learned")
    do, lwo, lso, _ = ni.net_values(pq, feats, d0, lw0, ls0)
    for got, ref, base in ((d, do, d0), (lw, lwo, lw0), (ls, lso, ls0)):
        nz = base != 0
        yg, yo = got[nz] / base[nz], ref[nz] / base[nz]
        assert np.max(np.abs(yg - yo)) <= 2e-2 * np.max(np.abs(yo - 1.0)) + 1e-6
    assert np.allclose(Z, ni.apply_P(d, lw, ls, k, 3, R), rtol=1e-12, atol=1e-12 * np.abs(Z).max())
    # loss and gradient over the pairs (M (-X) = B)
    loss, grad = e.net_grad(flat, B, X)
    L, g = ni.net_loss_and_grad(pq, feats, d0, lw0, ls0, k, 3, M, B, -X)
    gf = _flat({key: g[key] for key in ("w1", "b1", "w2", "b2", "w3", "b3")}).astype(np.float64)
    assert abs(loss - L) <= 1e-2 * abs(L)
    cos = float(grad @ gf) / (np.linalg.norm(grad) * np.linalg.norm(gf))
    assert cos >= 0.999, cos
    assert abs(np.linalg.norm(grad) / np.linalg.norm(gf) - 1.0) <= 3e-2
    # each layer's block separately (the tensor-core layer is w2, b2)
    off = 0
    for key in ("w1", "b1", "w2", "b2", "w3", "b3"):
        sz = g[key].size
        a, b = grad[off:off + sz], gf[off:off + sz]
        c = float(a @ b) / (np.linalg.norm(a) * np.linalg.norm(b))
        assert c >= 0.995, (key, c)
        off += sz
    e.close()


def test_learned_preconditioner_gains_over_ic0(pkg):
    k = 64
    A = _vc2d(k, 1000, corr=16.0)
    C = wl.rhs(A.shape[0], 2, 0)
    runs = {}
    for prec in ("jacobi", "ic0", "learned"):
        e = pkg.ExtendedKrylov(A, C, tol=1e-8, maxit=60, inner_tol=1e-10, grid=(k, k))
        st = e.solve(prec, train_solves=1, train_iters=150, lr=3e-3)
        assert st == 0
        runs[prec] = (e.m, e.history(), e.stats())
        e.close()
    (mj, hj, sj), (mi, hi, si), (ml, hl, sl) = runs["jacobi"], runs["ic0"], runs["learned"]
    assert mj == mi == ml
    assert np.all(np.abs(hl - hi) <= 1e-6 * np.abs(hi) + 1e-12)
    assert sl["network_accepted"] and sl["loss_after"] < sl["loss_before"]
    assert sl["inner_kinds"][0] == 1 and all(kd == 2 for kd in sl["inner_kinds"][1:]) and sl["fallbacks"] == 0
    it_j = sum(sj["inner_iterations"][1:])
    it_i = sum(si["inner_iterations"][1:])
    it_l = sum(sl["inner_iterations"][1:])
    print(f"inner CG iterations after the first solve: Jacobi {it_j}, IC(0) {it_i}, learned {it_l} "
          f"({it_l / it_i:.3f} of IC(0)); loss {sl['loss_before']:.4f} -> {sl['loss_after']:.4f}")
    assert it_i < it_j
    assert it_l <= 0.95 * it_i


def test_check_cuts_long_chains_of_resolved_eigenvalues(pkg):
    """The extended space resolves the small eigenvalues of a high-contrast operator early: at
    256^2 (sigma 1.5) T_m holds eigenvalues -19.4 ... -300 with gaps of 10 to 40 against ||T|| of
    4e7, closer than the fp64 grouping floor (1e-6 ||T||) yet resolved in fp64.  They chain into
    more members than one subspace iteration takes, and the chain is cut into consecutive groups:
    every m's history must equal the oracle's Prop. 3.1 evaluated on the GPU's own T_m."""
    import scipy.linalg as sla

    from oracle import lyap as olyap
    from paper_1602_05033_gb300 import _lib as L

    k = 256
    A = _vc2d(k, 1000, corr=8.0)
    C = wl.rhs(A.shape[0], 2, 0)
    beta = np.linalg.norm(C)
    e = pkg.ExtendedKrylov(A, C, tol=1e-8, maxit=18, inner_tol=1e-10, grid=(k, k))
    st = e.solve("ic0")
    assert st in (0, 1)
    h = e.history()
    longest = 0
    for m in range(1, len(h) + 1):
        ab, gam, tau = L.lyap_ek_projected_matrix(e.h, m, 4)
        lam, Q = sla.eig_banded(ab, lower=True)
        assert lam.max() < 0
        ref = olyap.cheap_residual(lam, Q, gam, tau, 4) / beta**2
        assert abs(h[m - 1] - ref) <= 1e-10 * ref + 1e-14, (m, h[m - 1], ref)
        close = np.diff(lam) <= 1e-6 * np.abs(lam).max()
        run = best = 0
        for c in close:
            run = run + 1 if c else 0
            best = max(best, run)
        longest = max(longest, best + 1)
    print("longest chain of estimates within the fp64 grouping floor:", longest)
    assert longest > 16  # the case this test is for
    e.close()
