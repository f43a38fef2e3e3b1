"""ctypes binding of liblyap.so: the C ABI of include/lyap.h, one Python function per entry point.

Only argument marshalling happens here; every step of the method runs in the
library's CUDA kernels.  Loading fails loudly when the library is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblyap.so")

LYAP_OK = 0
LYAP_NOT_CONVERGED = 1
LYAP_ERR_ARG = 2
LYAP_ERR_NONFINITE = 3
LYAP_ERR_BREAKDOWN = 4
LYAP_ERR_NOT_NEGDEF = 5
LYAP_ERR_TCAP = 6
LYAP_ERR_TIMEOUT = 7
LYAP_ERR_CUDA = 8
LYAP_ERR_WORKSPACE = 9
LYAP_ERR_EIGEN = 10

LYAP_F64, LYAP_F32 = 0, 1
LYAP_MEM_DEVICE, LYAP_MEM_HOST = 0, 1
LYAP_PREC_F64, LYAP_PREC_MIXED, LYAP_PREC_F32X2 = 0, 1, 2
LYAP_CHECK_ADAPTIVE = -1

# every symbol include/lyap.h declares
EXPORTED = (
    "lyap_default_options",
    "lyap_workspace_size",
    "lyap_create",
    "lyap_smallb_workspace_size",
    "lyap_smallb_create",
    "lyap_solve",
    "lyap_residual_norm",
    "lyap_factor",
    "lyap_projected_matrix",
    "lyap_phase_times",
    "lyap_destroy",
    "lyap_status_string",
    "lyap_residual_noalloc",
    "lyap_batch_workspace_size",
    "lyap_batch_create",
    "lyap_batch_solve",
    "lyap_batch_status",
    "lyap_batch_residual_norm",
    "lyap_batch_factor",
    "lyap_batch_tuning",
    "lyap_batch_phase_times",
    "lyap_batch_destroy",
    "lyap_ek_workspace_size",
    "lyap_ek_create",
    "lyap_ek_solve",
    "lyap_ek_residual_norm",
    "lyap_ek_factor",
    "lyap_ek_stats",
    "lyap_ek_net_grad",
    "lyap_ek_precond_apply",
    "lyap_ek_precond_values",
    "lyap_ek_precond_status",
    "lyap_ek_param_count",
    "lyap_ek_projected_matrix",
    "lyap_ek_destroy",
    "lyap_gen_workspace_size",
    "lyap_gen_create",
    "lyap_gen_solve",
    "lyap_gen_residual_norm",
    "lyap_gen_factor",
    "lyap_gen_stats",
    "lyap_gen_destroy",
)


class lyap_csr(ct.Structure):
    _fields_ = [
        ("n", ct.c_int64),
        ("nnz", ct.c_int64),
        ("rowptr", ct.c_void_p),
        ("col", ct.c_void_p),
        ("val", ct.c_void_p),
        ("val_dtype", ct.c_int),
        ("mem", ct.c_int),
    ]


class lyap_options(ct.Structure):
    _fields_ = [
        ("maxit", ct.c_int),
        ("check_every", ct.c_int),
        ("trunc_eps", ct.c_double),
        ("precision", ct.c_int),
        ("sell_sigma", ct.c_int),
        ("pass2_blocks", ct.c_int),
        ("check_batch", ct.c_int),
        ("zcap", ct.c_int),
    ]


class LyapError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


_lib = None


def load(path: str | None = None) -> ct.CDLL:
    """Loads liblyap.so (built by paper_1602_05033_gb300.build); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(the solver has no CPU fallback)"
        )
    lib = ct.CDLL(p)
    P = ct.c_void_p
    lib.lyap_default_options.argtypes = [ct.POINTER(lyap_options)]
    lib.lyap_default_options.restype = None
    lib.lyap_workspace_size.argtypes = [ct.POINTER(lyap_csr), ct.POINTER(lyap_csr), ct.c_int,
                                        ct.POINTER(lyap_options), ct.POINTER(ct.c_size_t)]
    lib.lyap_create.argtypes = [ct.POINTER(lyap_csr), ct.POINTER(lyap_csr), P, P, ct.c_int, ct.c_int, ct.c_double,
                                ct.POINTER(lyap_options), P, ct.c_size_t, P, ct.POINTER(P)]
    lib.lyap_smallb_workspace_size.argtypes = [ct.POINTER(lyap_csr), ct.c_int, ct.c_int, ct.POINTER(lyap_options),
                                                ct.POINTER(ct.c_size_t)]
    lib.lyap_smallb_create.argtypes = [ct.POINTER(lyap_csr), P, ct.c_int, P, P, ct.c_int, ct.c_int, ct.c_double,
                                       ct.POINTER(lyap_options), P, ct.c_size_t, P, ct.POINTER(P)]
    lib.lyap_solve.argtypes = [P, P]
    lib.lyap_residual_norm.argtypes = [P, ct.POINTER(ct.c_double), ct.c_int, ct.POINTER(ct.c_int)]
    lib.lyap_factor.argtypes = [P, P, ct.c_int64, P, ct.c_int64, ct.c_int, ct.c_int, ct.c_int,
                                ct.POINTER(ct.c_int), P]
    lib.lyap_projected_matrix.argtypes = [P, ct.c_int, ct.c_int, P, ct.c_int, P, P]
    lib.lyap_phase_times.argtypes = [P, ct.POINTER(ct.c_double), ct.c_int]
    lib.lyap_destroy.argtypes = [P]
    lib.lyap_residual_noalloc.argtypes = [ct.c_int, ct.c_int, P, ct.c_int, P, P, ct.c_double, P, P, P]
    CSRP = ct.POINTER(lyap_csr)
    IP = ct.POINTER(ct.c_int)
    lib.lyap_batch_workspace_size.argtypes = [ct.c_int, CSRP, IP, ct.POINTER(lyap_options), ct.POINTER(ct.c_size_t)]
    lib.lyap_batch_create.argtypes = [ct.c_int, CSRP, ct.POINTER(ct.c_void_p), ct.c_int, IP, ct.POINTER(ct.c_double),
                                      ct.POINTER(lyap_options), P, ct.c_size_t, P, ct.POINTER(P)]
    lib.lyap_batch_solve.argtypes = [P, ct.c_int, P]
    lib.lyap_batch_status.argtypes = [P, IP, IP]
    lib.lyap_batch_residual_norm.argtypes = [P, ct.c_int, ct.POINTER(ct.c_double), ct.c_int, IP]
    lib.lyap_batch_factor.argtypes = [P, ct.c_int, P, ct.c_int64, ct.c_int, ct.c_int, IP, P]
    lib.lyap_batch_tuning.argtypes = [P, IP, ct.c_int]
    lib.lyap_batch_phase_times.argtypes = [P, ct.POINTER(ct.c_double), ct.c_int]
    lib.lyap_batch_destroy.argtypes = [P]
    DP = ct.POINTER(ct.c_double)
    lib.lyap_ek_workspace_size.argtypes = [CSRP, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.POINTER(ct.c_size_t)]
    lib.lyap_ek_create.argtypes = [CSRP, P, ct.c_int, ct.c_int, ct.c_double, ct.c_int, ct.c_double, ct.c_int, ct.c_int, P,
                                   ct.c_size_t, P, ct.POINTER(P)]
    lib.lyap_ek_solve.argtypes = [P, ct.c_int, ct.c_int, ct.c_int, ct.c_float, P]
    lib.lyap_ek_residual_norm.argtypes = [P, DP, ct.c_int, IP]
    lib.lyap_ek_factor.argtypes = [P, P, ct.c_int64, ct.c_int, IP, P]
    lib.lyap_ek_stats.argtypes = [P, DP, ct.c_int]
    lib.lyap_ek_net_grad.argtypes = [P, ct.POINTER(ct.c_float), ct.c_int, P, P, DP, DP, P]
    lib.lyap_ek_precond_apply.argtypes = [P, ct.c_int, ct.POINTER(ct.c_float), ct.c_int, P, P, P]
    lib.lyap_ek_precond_values.argtypes = [P, ct.c_int, DP, DP, DP]
    lib.lyap_ek_precond_status.argtypes = [P]
    lib.lyap_ek_param_count.argtypes = []
    lib.lyap_ek_projected_matrix.argtypes = [P, ct.c_int, P, ct.c_int, P, P]
    lib.lyap_ek_destroy.argtypes = [P]
    lib.lyap_gen_workspace_size.argtypes = [CSRP, CSRP, ct.c_int, ct.c_int, ct.POINTER(ct.c_size_t)]
    lib.lyap_gen_create.argtypes = [CSRP, CSRP, P, ct.c_int, ct.c_int, ct.c_double, ct.c_int, ct.c_double, P,
                                    ct.c_size_t, P, ct.POINTER(P)]
    lib.lyap_gen_solve.argtypes = [P, P]
    lib.lyap_gen_residual_norm.argtypes = [P, DP, ct.c_int, IP]
    lib.lyap_gen_factor.argtypes = [P, P, ct.c_int64, ct.c_int, IP, P]
    lib.lyap_gen_stats.argtypes = [P, DP, ct.c_int]
    lib.lyap_gen_destroy.argtypes = [P]
    lib.lyap_status_string.argtypes = [ct.c_int]
    lib.lyap_status_string.restype = ct.c_char_p
    for name in EXPORTED:
        if name not in ("lyap_default_options", "lyap_status_string"):
            getattr(lib, name).restype = ct.c_int
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().lyap_status_string(int(status)).decode()


def lyap_default_options() -> lyap_options:
    o = lyap_options()
    load().lyap_default_options(ct.byref(o))
    return o


def lyap_workspace_size(A: lyap_csr, B: lyap_csr | None, s: int, opt: lyap_options | None) -> int:
    nb = ct.c_size_t(0)
    st = load().lyap_workspace_size(ct.byref(A), ct.byref(B) if B is not None else None, int(s),
                                    ct.byref(opt) if opt is not None else None, ct.byref(nb))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_workspace_size")
    return int(nb.value)


def lyap_create(A, B, C1_ptr: int, C2_ptr: int | None, c_mem: int, s: int, tol: float, opt, ws_ptr: int,
                ws_bytes: int, stream: int) -> int:
    h = ct.c_void_p(0)
    st = load().lyap_create(ct.byref(A), ct.byref(B) if B is not None else None, ct.c_void_p(C1_ptr),
                            ct.c_void_p(C2_ptr) if C2_ptr else None, int(c_mem), int(s), float(tol),
                            ct.byref(opt) if opt is not None else None, ct.c_void_p(ws_ptr), ct.c_size_t(ws_bytes),
                            ct.c_void_p(stream), ct.byref(h))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_create")
    return h.value


def lyap_smallb_workspace_size(A: lyap_csr, n2: int, s: int, opt: lyap_options | None) -> int:
    nb = ct.c_size_t(0)
    st = load().lyap_smallb_workspace_size(ct.byref(A), int(n2), int(s), ct.byref(opt) if opt is not None else None,
                                           ct.byref(nb))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_smallb_workspace_size")
    return int(nb.value)


def lyap_smallb_create(A, B_ptr: int, n2: int, C1_ptr: int, C2_ptr: int, c_mem: int, s: int, tol: float, opt,
                       ws_ptr: int, ws_bytes: int, stream: int) -> int:
    h = ct.c_void_p(0)
    st = load().lyap_smallb_create(ct.byref(A), ct.c_void_p(B_ptr), int(n2), ct.c_void_p(C1_ptr), ct.c_void_p(C2_ptr),
                                   int(c_mem), int(s), float(tol), ct.byref(opt) if opt is not None else None,
                                   ct.c_void_p(ws_ptr), ct.c_size_t(ws_bytes), ct.c_void_p(stream), ct.byref(h))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_smallb_create")
    return h.value


def lyap_solve(h: int, stream: int) -> int:
    st = load().lyap_solve(ct.c_void_p(h), ct.c_void_p(stream))
    if st not in (LYAP_OK, LYAP_NOT_CONVERGED):
        raise LyapError(st, "lyap_solve")
    return st


def lyap_residual_norm(h: int, cap: int):
    import numpy as np

    buf = np.full(max(cap, 1), np.nan)
    m = ct.c_int(0)
    st = load().lyap_residual_norm(ct.c_void_p(h), buf.ctypes.data_as(ct.POINTER(ct.c_double)), int(cap), ct.byref(m))
    if st not in (LYAP_OK, LYAP_NOT_CONVERGED):
        raise LyapError(st, "lyap_residual_norm")
    return buf[: m.value].copy(), m.value, st


def lyap_factor(h: int, Z1_ptr: int, ldz1: int, Z2_ptr: int | None, ldz2: int, z_dtype: int, z_mem: int, tcap: int,
                stream: int) -> int:
    t = ct.c_int(0)
    st = load().lyap_factor(ct.c_void_p(h), ct.c_void_p(Z1_ptr), ct.c_int64(ldz1),
                            ct.c_void_p(Z2_ptr) if Z2_ptr else None, ct.c_int64(ldz2), int(z_dtype), int(z_mem),
                            int(tcap), ct.byref(t), ct.c_void_p(stream))
    if st != LYAP_OK:
        err = LyapError(st, "lyap_factor")
        err.t = t.value
        raise err
    return t.value


def lyap_projected_matrix(h: int, op: int, m: int, s: int):
    """(ab, gamma, tau_next): T_m in lower band storage ab[d, i] = T_m[i+d, i], and the s x s blocks."""
    import numpy as np

    N = s * m
    ab = np.zeros((N, s + 1))
    gam = np.zeros((s, s))
    tau = np.zeros((s, s))
    st = load().lyap_projected_matrix(ct.c_void_p(h), int(op), int(m), ab.ctypes.data, s + 1, gam.ctypes.data,
                                      tau.ctypes.data)
    if st != LYAP_OK:
        raise LyapError(st, "lyap_projected_matrix")
    return np.ascontiguousarray(ab.T), gam, tau


def lyap_phase_times(h: int):
    out = (ct.c_double * 10)()
    load().lyap_phase_times(ct.c_void_p(h), out, 10)
    return list(out)


def lyap_residual_noalloc(s: int, m: int, ab_ptr: int, ldab: int, gamma_ptr: int, tau_ptr: int, beta: float,
                          rel_ptr: int, status_ptr: int, stream: int) -> None:
    """Enqueues the allocation-free residual evaluation; all pointers are device memory."""
    st = load().lyap_residual_noalloc(int(s), int(m), ct.c_void_p(ab_ptr), int(ldab), ct.c_void_p(gamma_ptr),
                                      ct.c_void_p(tau_ptr), float(beta), ct.c_void_p(rel_ptr), ct.c_void_p(status_ptr),
                                      ct.c_void_p(stream))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_residual_noalloc")


def _arr(ctype, vals):
    return (ctype * len(vals))(*vals)


def lyap_batch_workspace_size(csrs, s, opt) -> int:
    nb = ct.c_size_t(0)
    st = load().lyap_batch_workspace_size(len(csrs), _arr(lyap_csr, csrs), _arr(ct.c_int, s),
                                          ct.byref(opt) if opt is not None else None, ct.byref(nb))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_batch_workspace_size")
    return int(nb.value)


def lyap_batch_create(csrs, c_ptrs, c_mem: int, s, tol, opt, ws_ptr: int, ws_bytes: int, stream: int) -> int:
    h = ct.c_void_p(0)
    st = load().lyap_batch_create(len(csrs), _arr(lyap_csr, csrs), _arr(ct.c_void_p, c_ptrs), int(c_mem),
                                  _arr(ct.c_int, s), _arr(ct.c_double, tol),
                                  ct.byref(opt) if opt is not None else None, ct.c_void_p(ws_ptr),
                                  ct.c_size_t(ws_bytes), ct.c_void_p(stream), ct.byref(h))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_batch_create")
    return h.value


def lyap_batch_solve(b: int, autotune: bool, stream: int) -> int:
    """Returns the batch status; an instance's own failure (breakdown, eigensolver, ...) is
    reported through lyap_batch_status, only failures of the call itself raise."""
    st = load().lyap_batch_solve(ct.c_void_p(b), int(bool(autotune)), ct.c_void_p(stream))
    if st in (LYAP_ERR_ARG, LYAP_ERR_CUDA, LYAP_ERR_WORKSPACE):
        raise LyapError(st, "lyap_batch_solve")
    return st


def lyap_batch_status(b: int, count: int):
    stt = (ct.c_int * count)()
    m = (ct.c_int * count)()
    st = load().lyap_batch_status(ct.c_void_p(b), stt, m)
    if st != LYAP_OK:
        raise LyapError(st, "lyap_batch_status")
    return list(stt), list(m)


def lyap_batch_residual_norm(b: int, i: int, cap: int):
    import numpy as np

    buf = np.full(max(cap, 1), np.nan)
    m = ct.c_int(0)
    st = load().lyap_batch_residual_norm(ct.c_void_p(b), int(i), buf.ctypes.data_as(ct.POINTER(ct.c_double)), int(cap),
                                         ct.byref(m))
    if st not in (LYAP_OK, LYAP_NOT_CONVERGED):
        raise LyapError(st, "lyap_batch_residual_norm")
    return buf[: m.value].copy(), m.value


def lyap_batch_factor(b: int, i: int, Z_ptr: int, ldz: int, z_dtype: int, tcap: int, stream: int) -> int:
    t = ct.c_int(0)
    st = load().lyap_batch_factor(ct.c_void_p(b), int(i), ct.c_void_p(Z_ptr), ct.c_int64(ldz), int(z_dtype), int(tcap),
                                  ct.byref(t), ct.c_void_p(stream))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_batch_factor")
    return t.value


def lyap_batch_tuning(b: int):
    out = (ct.c_int * 48)()
    n = load().lyap_batch_tuning(ct.c_void_p(b), out, 48)
    return [tuple(out[3 * g:3 * g + 3]) for g in range(max(n, 0))]


def lyap_batch_phase_times(b: int):
    out = (ct.c_double * 8)()
    load().lyap_batch_phase_times(ct.c_void_p(b), out, 8)
    return list(out)


def lyap_batch_destroy(b: int) -> None:
    if b:
        load().lyap_batch_destroy(ct.c_void_p(b))


def lyap_ek_workspace_size(A: lyap_csr, s: int, maxit: int, nx: int, ny: int) -> int:
    nb = ct.c_size_t(0)
    st = load().lyap_ek_workspace_size(ct.byref(A), int(s), int(maxit), int(nx), int(ny), ct.byref(nb))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_ek_workspace_size")
    return int(nb.value)


def lyap_ek_create(A: lyap_csr, C_ptr: int, c_mem: int, s: int, tol: float, maxit: int, inner_tol: float, nx: int,
                   ny: int, ws_ptr: int, ws_bytes: int, stream: int) -> int:
    h = ct.c_void_p(0)
    st = load().lyap_ek_create(ct.byref(A), ct.c_void_p(C_ptr), int(c_mem), int(s), float(tol), int(maxit),
                               float(inner_tol), int(nx), int(ny), ct.c_void_p(ws_ptr), ct.c_size_t(ws_bytes),
                               ct.c_void_p(stream), ct.byref(h))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_ek_create")
    return h.value


def lyap_ek_solve(h: int, precond: int, train_steps: int, train_iters: int, lr: float, stream: int) -> int:
    st = load().lyap_ek_solve(ct.c_void_p(h), int(precond), int(train_steps), int(train_iters), float(lr),
                              ct.c_void_p(stream))
    if st not in (LYAP_OK, LYAP_NOT_CONVERGED):
        raise LyapError(st, "lyap_ek_solve")
    return st


def lyap_ek_residual_norm(h: int, cap: int):
    import numpy as np

    buf = np.full(max(cap, 1), np.nan)
    m = ct.c_int(0)
    st = load().lyap_ek_residual_norm(ct.c_void_p(h), buf.ctypes.data_as(ct.POINTER(ct.c_double)), int(cap), ct.byref(m))
    if st not in (LYAP_OK, LYAP_NOT_CONVERGED):
        raise LyapError(st, "lyap_ek_residual_norm")
    return buf[: m.value].copy(), m.value


def lyap_ek_factor(h: int, Z_ptr: int, ldz: int, tcap: int, stream: int) -> int:
    t = ct.c_int(0)
    st = load().lyap_ek_factor(ct.c_void_p(h), ct.c_void_p(Z_ptr), ct.c_int64(ldz), int(tcap), ct.byref(t),
                               ct.c_void_p(stream))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_ek_factor")
    return t.value


def lyap_ek_stats(h: int, cap: int = 512):
    out = (ct.c_double * cap)()
    load().lyap_ek_stats(ct.c_void_p(h), out, cap)
    return list(out)


def lyap_ek_param_count() -> int:
    return int(load().lyap_ek_param_count())


def lyap_ek_net_grad(h: int, params, K: int, B_ptr: int, X_ptr: int, stream: int):
    import numpy as np

    nw = lyap_ek_param_count()
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == nw
    loss = ct.c_double(0.0)
    grad = np.zeros(nw)
    st = load().lyap_ek_net_grad(ct.c_void_p(h), p.ctypes.data_as(ct.POINTER(ct.c_float)), int(K), ct.c_void_p(B_ptr),
                                 ct.c_void_p(X_ptr), ct.byref(loss), grad.ctypes.data_as(ct.POINTER(ct.c_double)),
                                 ct.c_void_p(stream))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_ek_net_grad")
    return loss.value, grad


def lyap_ek_precond_apply(h: int, kind: int, params, K: int, R_ptr: int, Z_ptr: int, stream: int) -> None:
    import numpy as np

    pp = None
    if params is not None:
        arr = np.ascontiguousarray(params, dtype=np.float32)
        assert arr.size == lyap_ek_param_count()
        pp = arr.ctypes.data_as(ct.POINTER(ct.c_float))
    st = load().lyap_ek_precond_apply(ct.c_void_p(h), int(kind), pp, int(K), ct.c_void_p(R_ptr), ct.c_void_p(Z_ptr),
                                      ct.c_void_p(stream))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_ek_precond_apply")


def lyap_ek_precond_values(h: int, kind: int, n: int):
    import numpy as np

    d, lw, ls = np.zeros(n), np.zeros(n), np.zeros(n)
    st = load().lyap_ek_precond_values(ct.c_void_p(h), int(kind), *(a.ctypes.data_as(ct.POINTER(ct.c_double))
                                                                      for a in (d, lw, ls)))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_ek_precond_values")
    return d, lw, ls


def lyap_ek_precond_status(h: int) -> int:
    return int(load().lyap_ek_precond_status(ct.c_void_p(h)))


def lyap_ek_projected_matrix(h: int, m: int, S: int):
    """(ab, gamma, tau_next) of the extended space's T_m: ab is (S+1) x (S*m) lower band storage."""
    import numpy as np

    N = S * m
    ab = np.zeros((N, S + 1))
    gam = np.zeros((S, S))
    tau = np.zeros((S, S))
    st = load().lyap_ek_projected_matrix(ct.c_void_p(h), int(m), ab.ctypes.data, S + 1, gam.ctypes.data, tau.ctypes.data)
    if st != LYAP_OK:
        raise LyapError(st, "lyap_ek_projected_matrix")
    return ab.T.copy(), gam, tau


def lyap_ek_destroy(h: int) -> None:
    if h:
        load().lyap_ek_destroy(ct.c_void_p(h))


def lyap_destroy(h: int) -> None:
    if h:
        load().lyap_destroy(ct.c_void_p(h))


def lyap_gen_workspace_size(A: lyap_csr, E: lyap_csr, s: int, maxit: int) -> int:
    nb = ct.c_size_t(0)
    st = load().lyap_gen_workspace_size(ct.byref(A), ct.byref(E), int(s), int(maxit), ct.byref(nb))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_gen_workspace_size")
    return int(nb.value)


def lyap_gen_create(A: lyap_csr, E: lyap_csr, C_ptr: int, c_mem: int, s: int, tol: float, maxit: int,
                    inner_tol: float, ws_ptr: int, ws_bytes: int, stream: int) -> int:
    h = ct.c_void_p(0)
    st = load().lyap_gen_create(ct.byref(A), ct.byref(E), ct.c_void_p(C_ptr), int(c_mem), int(s), float(tol),
                                int(maxit), float(inner_tol), ct.c_void_p(ws_ptr), ct.c_size_t(ws_bytes),
                                ct.c_void_p(stream), ct.byref(h))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_gen_create")
    return h.value


def lyap_gen_solve(h: int, stream: int) -> int:
    st = load().lyap_gen_solve(ct.c_void_p(h), ct.c_void_p(stream))
    if st not in (LYAP_OK, LYAP_NOT_CONVERGED):
        raise LyapError(st, "lyap_gen_solve")
    return st


def lyap_gen_residual_norm(h: int, cap: int):
    import numpy as np

    buf = np.full(max(cap, 1), np.nan)
    m = ct.c_int(0)
    st = load().lyap_gen_residual_norm(ct.c_void_p(h), buf.ctypes.data_as(ct.POINTER(ct.c_double)), int(cap),
                                       ct.byref(m))
    if st not in (LYAP_OK, LYAP_NOT_CONVERGED):
        raise LyapError(st, "lyap_gen_residual_norm")
    return buf[: m.value].copy(), m.value


def lyap_gen_factor(h: int, Z_ptr: int, ldz: int, tcap: int, stream: int) -> int:
    t = ct.c_int(0)
    st = load().lyap_gen_factor(ct.c_void_p(h), ct.c_void_p(Z_ptr), ct.c_int64(ldz), int(tcap), ct.byref(t),
                                ct.c_void_p(stream))
    if st != LYAP_OK:
        raise LyapError(st, "lyap_gen_factor")
    return t.value


def lyap_gen_stats(h: int):
    out = (ct.c_double * 4)()
    load().lyap_gen_stats(ct.c_void_p(h), out, 4)
    return list(out)


def lyap_gen_destroy(h: int) -> None:
    if h:
        load().lyap_gen_destroy(ct.c_void_p(h))
