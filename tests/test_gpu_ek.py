"""GPU parity of the extended Krylov path (Sec. 4) and of the learned preconditioner's kernels.

  * EK with conjugate-gradient inner solves (inner tolerance 1e-13) against the FP64 oracle with
    exact solves: the same iteration count and histories within 1e-9 rel. (+1e-12), the factor
    by X probes;
  * the network's energy-norm loss and gradient (bf16 activations, fp32 accumulation) against
    the fp64 oracle evaluated with the same bf16-rounded weights;
  * training on the method's own solve pairs lowers the loss, and the trained network keeps the
    method's result while its inner iterations are compared with Jacobi's.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import cnn as ocnn
from oracle import ek as oek

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


def _xprobe(Z, Zo, seed=0):
    u = np.random.default_rng(seed).standard_normal((Z.shape[0], 3))
    a = Z @ (Z.T @ u)
    b = Zo @ (Zo.T @ u)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name,mk,s", [("lap2d20_s1", lambda: wl.laplacian_2d(20), 1),
                                       ("vc2d16_s2", lambda: _vc2d(16, 3), 2),
                                       ("lap2d12_s4", lambda: wl.laplacian_2d(12), 4)])
def test_ek_matches_oracle(pkg, name, mk, s):
    A = mk()
    C = wl.rhs(A.shape[0], s, 9)
    ref = oek.solve(A, C, tol=1e-9, maxit=40)
    e = pkg.ExtendedKrylov(A, C, tol=1e-9, maxit=40, inner_tol=1e-13)
    st = e.solve("jacobi")
    assert st == 0 and e.m == ref.m
    h = e.history()
    assert np.all(np.abs(h - ref.history) <= 1e-12 + 1e-9 * np.abs(ref.history)), np.max(np.abs(h - ref.history))
    Z = e.factor().cpu().numpy()
    Zo, _ = oek.factor(ref)
    assert _xprobe(Z, Zo) <= 1e-7
    e.close()


def _flat(p):
    return np.concatenate([p["w1"].ravel(), p["b1"], p["w2"].ravel(), p["b2"], p["w3"].ravel(), p["b3"]]).astype(np.float32)


def _unflat(v, C=16):
    k = 0
    out = {}
    for key, shape in (("w1", (C, 1, 3, 3)), ("b1", (C,)), ("w2", (C, C, 3, 3)), ("b2", (C,)), ("w3", (1, C, 3, 3)),
                       ("b3", (1,))):
        sz = int(np.prod(shape))
        out[key] = np.asarray(v[k:k + sz], dtype=np.float64).reshape(shape)
        k += sz
    return out


def _bf16(v):
    """Round float32 values to bfloat16 (round to nearest even), back to float64."""
    u = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_cnn_gradient_matches_oracle(pkg):
    ny = nx = 12
    kappa = np.exp(wl.gaussian_field(12, 2, seed=7, corr_len=3.0))
    A = wl.var_coeff_diffusion(kappa)  # 12 x 12 grid
    n = A.shape[0]
    rng = np.random.default_rng(1)
    X = rng.standard_normal((n, 2))
    B = A @ X
    p = ocnn.init_params(C=16, seed=4, scale=0.3)
    flat = _flat(p)
    e = pkg.ExtendedKrylov(A, rng.standard_normal((n, 1)), maxit=4, grid=(nx, ny))
    loss, grad = e.cnn_grad(flat, B, X)
    # the oracle with the weights the kernels use (bf16) and fp64 activations
    pq = _unflat(_bf16(flat))
    for key in ("b1", "b2", "b3"):
        pq[key] = _unflat(flat)[key]  # biases stay fp32
    L, g = ocnn.energy_loss_and_grad(pq, A, B, X, (ny, nx), jacobi=True)
    gf = _flat({k: g[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3")}).astype(np.float64)
    assert abs(loss - L) <= 2e-2 * abs(L)
    cos = float(grad @ gf) / (np.linalg.norm(grad) * np.linalg.norm(gf))
    assert cos >= 0.999, cos
    assert abs(np.linalg.norm(grad) / np.linalg.norm(gf) - 1.0) <= 3e-2
    e.close()


def test_trained_network_as_preconditioner(pkg):
    k = 32
    A = _vc2d(k, 11, sigma=1.5, corr=6.0)
    C = wl.rhs(A.shape[0], 2, 3)
    jac = pkg.ExtendedKrylov(A, C, tol=1e-8, maxit=40, inner_tol=1e-10, grid=(k, k))
    jac.solve("jacobi")
    net = pkg.ExtendedKrylov(A, C, tol=1e-8, maxit=40, inner_tol=1e-10, grid=(k, k))
    net.solve("cnn", train_steps=2, train_iters=300, lr=2e-3)
    sj, sn = jac.stats(), net.stats()
    print("inner iterations jacobi", sj["inner_jacobi"], "cnn", sn["inner_cnn"], "fallbacks", sn["fallbacks"],
          "loss", sn["loss_before"], sn["loss_after"])
    assert sn["loss_after"] < sn["loss_before"]
    assert net.m == jac.m
    hj, hn = jac.history(), net.history()
    assert np.all(np.abs(hj - hn) <= 1e-6 * np.abs(hj) + 1e-12)
    jac.close()
    net.close()
