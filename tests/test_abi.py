"""The C-ABI library loads and exports every symbol include/lyap.h declares (no GPU needed)."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

import workloads as wl


@pytest.fixture(scope="module")
def lib(repo_root):
    from paper_1602_05033_gb300 import _lib
    from paper_1602_05033_gb300 import build as b

    if not os.path.exists(_lib.LIB_PATH):
        b.build()
    return _lib.load()


def _declared(repo_root):
    text = open(os.path.join(repo_root, "include", "lyap.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lyap_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib, repo_root):
    from paper_1602_05033_gb300 import _lib

    names = _declared(repo_root)
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(_lib.EXPORTED) == names


def test_status_strings_and_defaults(lib):
    from paper_1602_05033_gb300 import _lib

    assert _lib.status_string(0) == "ok"
    assert "breakdown" in _lib.status_string(_lib.LYAP_ERR_BREAKDOWN).lower()
    o = _lib.lyap_default_options()
    assert o.maxit == 1000 and o.check_every == 1 and o.trunc_eps == 0.0 and o.pass2_blocks == 16
    assert o.precision == _lib.LYAP_PREC_F64 and _lib.LYAP_PREC_F32X2 == 2


def _host_csr(A, keep):
    from paper_1602_05033_gb300 import _lib, csr_arrays

    rp, cl, vl = csr_arrays(A)
    keep += [rp, cl, vl]
    c = _lib.lyap_csr()
    c.n, c.nnz = A.shape[0], cl.shape[0]
    c.rowptr, c.col, c.val = rp.ctypes.data, cl.ctypes.data, vl.ctypes.data
    c.val_dtype, c.mem = _lib.LYAP_F64, _lib.LYAP_MEM_HOST
    return c


def test_workspace_size_host_inputs(lib):
    """Host-side planning only: SELL padding and the storage of Alg. 1 grow as documented."""
    from paper_1602_05033_gb300 import _lib

    keep = []
    A = _host_csr(wl.laplacian_2d(30), keep)
    o = _lib.lyap_default_options()
    o.maxit = 100
    b1 = _lib.lyap_workspace_size(A, None, 1, o)
    b4 = _lib.lyap_workspace_size(A, None, 4, o)
    o.maxit = 200
    b4b = _lib.lyap_workspace_size(A, None, 4, o)
    assert 0 < b1 < b4 < b4b
    B = _host_csr(wl.laplacian_2d(20), keep)
    assert _lib.lyap_workspace_size(A, B, 4, o) > b4b


def test_invalid_arguments_rejected(lib):
    from paper_1602_05033_gb300 import _lib

    keep = []
    A = _host_csr(wl.laplacian_2d(8), keep)
    o = _lib.lyap_default_options()
    with pytest.raises(_lib.LyapError) as e:
        _lib.lyap_workspace_size(A, None, 5, o)  # unsupported block size
    assert e.value.status == _lib.LYAP_ERR_ARG
    bad = _lib.lyap_csr()
    bad.n = -1
    with pytest.raises(_lib.LyapError):
        _lib.lyap_workspace_size(bad, None, 1, o)
    # rowptr that does not end at nnz
    rp = np.array([0, 1, 3], dtype=np.int64)
    keep.append(rp)
    A2 = _lib.lyap_csr()
    A2.n, A2.nnz, A2.rowptr, A2.col, A2.val = 2, 2, rp.ctypes.data, rp.ctypes.data, rp.ctypes.data
    A2.val_dtype, A2.mem = _lib.LYAP_F64, _lib.LYAP_MEM_HOST
    with pytest.raises(_lib.LyapError):
        _lib.lyap_workspace_size(A2, None, 1, o)


def test_batch_planning_pools(lib):
    """Batched planning on the host: every instance adds its own storage, and each of the
    first twelve instances adds a pool (a check area of at least 2 GiB plus factor scratch)."""
    from paper_1602_05033_gb300 import _lib

    keep = []
    A = _host_csr(wl.laplacian_2d(16), keep)
    o = _lib.lyap_default_options()
    o.maxit = 50

    def size(c):
        return _lib.lyap_batch_workspace_size([A] * c, [2] * c, o)

    gib = 1 << 30
    s1, s2, s12, s13 = size(1), size(2), size(12), size(13)
    assert s2 - s1 >= 2 * gib  # the second instance brings a second pool
    assert s12 - size(11) >= 2 * gib
    assert 0 < s13 - s12 < 2 * gib  # no pool beyond twelve
    with pytest.raises(_lib.LyapError) as e:
        _lib.lyap_batch_workspace_size([A, A], [2, 5], o)
    assert e.value.status == _lib.LYAP_ERR_ARG
    o.sell_sigma = 4  # batched sweeps take the natural row order only
    with pytest.raises(_lib.LyapError) as e:
        _lib.lyap_batch_workspace_size([A], [2], o)
    assert e.value.status == _lib.LYAP_ERR_ARG


def test_ek_planning_rejects_bad_arguments(lib):
    from paper_1602_05033_gb300 import _lib

    keep = []
    A = _host_csr(wl.laplacian_2d(16), keep)
    assert _lib.lyap_ek_workspace_size(A, 2, 20, 16, 16) > _lib.lyap_ek_workspace_size(A, 2, 10, 16, 16) > 0
    # the grid adds the preconditioners' state: stencil, IC(0) and learned values, network
    # activations and the training blocks (19 blocks of n x 4 values of the Horner passes)
    n = 256
    extra = _lib.lyap_ek_workspace_size(A, 2, 20, 16, 16) - _lib.lyap_ek_workspace_size(A, 2, 20, 0, 0)
    assert extra >= 8 * n * (5 + 1 + 6 + 3 + 19 * 4 + 12) + 2 * n * 16 * 4
    for s, maxit, nx, ny in [(3, 20, 16, 16), (2, 0, 16, 16), (2, 20, 16, 15), (2, 20, -16, -16)]:
        with pytest.raises(_lib.LyapError) as e:
            _lib.lyap_ek_workspace_size(A, s, maxit, nx, ny)
        assert e.value.status == _lib.LYAP_ERR_ARG
    A.val_dtype = _lib.LYAP_F32  # the extended Krylov path is fp64
    with pytest.raises(_lib.LyapError) as e:
        _lib.lyap_ek_workspace_size(A, 2, 20, 16, 16)
    assert e.value.status == _lib.LYAP_ERR_ARG


def test_create_rejects_bad_arguments_before_any_device_work(lib):
    from paper_1602_05033_gb300 import _lib

    keep = []
    A = _host_csr(wl.laplacian_2d(8), keep)
    C = np.ones((64, 2))
    keep.append(C)
    o = _lib.lyap_default_options()
    cases = [
        dict(s=5, tol=1e-8, c_mem=_lib.LYAP_MEM_HOST, B=None),   # unsupported block size
        dict(s=2, tol=-1.0, c_mem=_lib.LYAP_MEM_HOST, B=None),   # negative tolerance
        dict(s=2, tol=1e-8, c_mem=7, B=None),                     # unknown memory kind
        dict(s=2, tol=1e-8, c_mem=_lib.LYAP_MEM_HOST, B=A),      # B without C2
    ]
    for c in cases:
        with pytest.raises(_lib.LyapError) as e:
            _lib.lyap_create(A, c["B"], C.ctypes.data, None, c["c_mem"], c["s"], c["tol"], o, 0, 0, 0)
        assert e.value.status == _lib.LYAP_ERR_ARG, c


def test_two_pass_storage_does_not_grow_with_n_times_m(lib):
    """The memory device of Sec. 3.3: the basis is not stored, so raising maxit adds
    only m-sized storage (coefficient log, history, check slots of the reduced problem), the same
    for a 4x larger operator; the n-sized part (three blocks, W, the pass-2 buffer, the operator
    copy) does not depend on maxit."""
    from paper_1602_05033_gb300 import _lib

    keep = []
    small = _host_csr(wl.laplacian_2d(60), keep)    # n = 3600
    large = _host_csr(wl.laplacian_2d(120), keep)   # n = 14400
    o = _lib.lyap_default_options()
    growth = []
    for A in (small, large):
        o.maxit = 100
        a = _lib.lyap_workspace_size(A, None, 4, o)
        o.maxit = 300
        b = _lib.lyap_workspace_size(A, None, 4, o)
        growth.append(b - a)
    # identical growth for a 4x larger operator: nothing of size n x m is stored (the reduced
    # problem's check slots, O((s m)^2), are what grows)
    assert growth[0] == growth[1] > 0
