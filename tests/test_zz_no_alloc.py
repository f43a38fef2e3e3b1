"""The allocation-free residual entry point (lyap_residual_noalloc) against lyap_solve and the oracle.

lyap_residual_noalloc serves callers that cannot allocate device memory when they need a
residual norm, for instance code running inside another framework whose caching allocator
already holds the free memory.  It evaluates the same residual as the convergence check of
lyap_solve, with its scratch in a fixed array inside the library.  This test feeds it the
projected matrices of a solve (exported by lyap_projected_matrix), calls it twice in a row
(the second call must not see anything the first left in the shared array) and compares the
results with the history lyap_solve recorded and with the FP64 oracle's residual formula on
the same T_m, within the tolerance of the check tests.  After a first call (which, with lazy
module loading, loads the library's device code and its array), further calls must leave the
device's free memory and the caching allocator's reservation unchanged.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import lyap as olyap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_05033_gb300 import _lib
    from paper_1602_05033_gb300 import build as b

    b.build()
    _lib.load()
    return torch, _lib


def test_noalloc_residual_matches_solve_history(env):
    torch, L = env
    from paper_1602_05033_gb300 import Solver

    A = wl.laplacian_2d(16)
    s = 2
    C = wl.rhs(A.shape[0], s, 3)
    sol = Solver(A, C, tol=1e-9, maxit=120)
    sol.solve()
    hist = sol.history()
    beta = float(np.linalg.norm(C))
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    rel = torch.zeros(1, dtype=torch.float64, device=dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    ms = [m for m in (sol.m, 7, sol.m // 2) if 1 <= m <= sol.m and s * m <= 256]
    for m in ms:
        ab, gam, tau = sol.projected(m)
        ab_d = torch.from_numpy(np.ascontiguousarray(ab.T)).to(dev)  # ab[d + i*(s+1)] layout
        gam_d = torch.from_numpy(np.ascontiguousarray(gam)).to(dev)
        tau_d = torch.from_numpy(np.ascontiguousarray(tau)).to(dev)
        for _ in range(2):  # two calls in a row share the same scratch
            rel.zero_()
            status.fill_(-1)
            L.lyap_residual_noalloc(s, m, ab_d.data_ptr(), s + 1, gam_d.data_ptr(), tau_d.data_ptr(), beta,
                                    rel.data_ptr(), status.data_ptr(), stream)
            torch.cuda.synchronize()
            assert int(status.item()) == L.LYAP_OK
            got = float(rel.item())
            ref = float(hist[m - 1])
            assert abs(got - ref) <= 1e-10 * ref + 1e-14, (m, got, ref)
            lam, Q = sla.eig_banded(ab, lower=True)
            ora = olyap.cheap_residual(lam, Q, gam, tau, s) / beta**2
            assert abs(got - ora) <= 1e-10 * ora + 1e-14, (m, got, ora)
    sol.close()


def test_noalloc_calls_allocate_nothing(env):
    torch, L = env
    from paper_1602_05033_gb300 import Solver

    A = wl.laplacian_2d(12)
    s = 3
    C = wl.rhs(A.shape[0], s, 5)
    sol = Solver(A, C, tol=1e-9, maxit=60)
    sol.solve()
    m = min(sol.m, 256 // s)
    ab, gam, tau = sol.projected(m)
    beta = float(np.linalg.norm(C))
    sol.close()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    ab_d = torch.from_numpy(np.ascontiguousarray(ab.T)).to(dev)
    gam_d = torch.from_numpy(np.ascontiguousarray(gam)).to(dev)
    tau_d = torch.from_numpy(np.ascontiguousarray(tau)).to(dev)
    rel = torch.zeros(1, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)

    def call():
        L.lyap_residual_noalloc(s, m, ab_d.data_ptr(), s + 1, gam_d.data_ptr(), tau_d.data_ptr(), beta,
                                rel.data_ptr(), status.data_ptr(), stream)

    call()  # set-up call: loads the device code and the array on this device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    res0 = torch.cuda.memory_reserved(dev)
    vals = []
    for _ in range(3):
        call()
        torch.cuda.synchronize()
        vals.append(float(rel.item()))
    free1, _ = torch.cuda.mem_get_info(dev)
    assert torch.cuda.memory_reserved(dev) == res0
    assert free1 == free0, (free0, free1)
    assert int(status.item()) == L.LYAP_OK
    assert vals[0] == vals[1] == vals[2]


def test_noalloc_rejects_sizes_beyond_its_array(env):
    torch, L = env
    dev = torch.device("cuda:0")
    buf = torch.zeros(64, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for s, m in ((2, 129), (5, 1), (4, 65)):
        with pytest.raises(L.LyapError) as e:
            L.lyap_residual_noalloc(s, m, buf.data_ptr(), s + 1, buf.data_ptr(), buf.data_ptr(), 1.0, buf.data_ptr(),
                                    st.data_ptr(), stream)
        assert e.value.status == L.LYAP_ERR_ARG
