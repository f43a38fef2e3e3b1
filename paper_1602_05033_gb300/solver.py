"""Convenience wrapper over the C ABI: PyTorch owns the device memory, liblyap does the work."""
from __future__ import annotations

import numpy as np

from . import _lib as L


def csr_arrays(A):
    """(rowptr int64, col int32, val float64) of a scipy CSR matrix, contiguous."""
    A = A.tocsr()
    return (np.ascontiguousarray(A.indptr, dtype=np.int64), np.ascontiguousarray(A.indices, dtype=np.int32),
            np.ascontiguousarray(A.data, dtype=np.float64))


# bulk number type of a solve: fp64, fp32 ("mixed": fp32 basis, float-pair sums), float pairs
PRECISIONS = {"f64": L.LYAP_PREC_F64, "mixed": L.LYAP_PREC_MIXED, "f32x2": L.LYAP_PREC_F32X2}


class Solver:
    """One Lyapunov (B is None) or Sylvester solve through lyap_create/solve/factor.

    A sparse B projects both operators (Sec. 5.1); a dense numpy B (small, n2 x n2) takes the
    large-A / small-B path of Sec. 5.2 through lyap_smallb_create.
    ``inputs="device"`` uploads A, B, C with PyTorch before calling lyap_create;
    ``inputs="host"`` hands host pointers to lyap_create, which copies them.
    """

    def __init__(self, A, C1, B=None, C2=None, *, tol=1e-8, maxit=1000, check_every=1, trunc_eps=0.0,
                 precision="f64", sell_sigma=1, pass2_blocks=16, check_batch=32, zcap=0, inputs="device",
                 device="cuda:0", val_dtype="f64"):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.sylv = B is not None
        self.small_b = isinstance(B, np.ndarray)
        self.s = int(C1.shape[1])
        self.n1 = int(A.shape[0])
        self.n2 = int(B.shape[0]) if self.sylv else self.n1
        self.precision = PRECISIONS[precision]
        self.maxit = int(maxit)
        opt = L.lyap_default_options()
        opt.maxit = int(maxit)
        opt.check_every = L.LYAP_CHECK_ADAPTIVE if check_every == "adaptive" else int(check_every)
        opt.trunc_eps = float(trunc_eps)
        opt.precision = self.precision
        opt.sell_sigma = int(sell_sigma)
        opt.pass2_blocks = int(pass2_blocks)
        opt.check_batch = int(check_batch)
        # host output of the factor is staged in the workspace; by default size it for any rank
        opt.zcap = int(zcap) if zcap else (self.s * int(maxit) if inputs == "host" else 0)
        self.opt = opt
        self._keep = []
        vdt = np.float32 if val_dtype == "f32" else np.float64
        self._csr = [self._make_csr(A, inputs, vdt)]
        if self.sylv and not self.small_b:
            self._csr.append(self._make_csr(B, inputs, vdt))
        if self.small_b:
            self.ws_bytes = L.lyap_smallb_workspace_size(self._csr[0], self.n2, self.s, opt)
        else:
            self.ws_bytes = L.lyap_workspace_size(self._csr[0], self._csr[1] if self.sylv else None, self.s, opt)
        with torch.cuda.device(self.device):
            self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device).cuda_stream
        c_mem = L.LYAP_MEM_HOST if inputs == "host" else L.LYAP_MEM_DEVICE
        cptr = [self._make_rhs(C1, inputs)]
        if self.sylv:
            cptr.append(self._make_rhs(C2, inputs))
        if self.small_b:
            bptr = self._make_rhs(B, inputs)
            self.h = L.lyap_smallb_create(self._csr[0], bptr, self.n2, cptr[0], cptr[1], c_mem, self.s, tol, opt,
                                          self.ws.data_ptr(), self.ws_bytes, self.stream)
        else:
            self.h = L.lyap_create(self._csr[0], self._csr[1] if self.sylv else None, cptr[0],
                                   cptr[1] if self.sylv else None, c_mem, self.s, tol, opt, self.ws.data_ptr(),
                                   self.ws_bytes, self.stream)
        self._keep.clear()
        self.status = None
        self.m = 0

    def _make_csr(self, A, inputs, vdt):
        rp, cl, vl = csr_arrays(A)
        vl = vl.astype(vdt)
        c = L.lyap_csr()
        c.n = A.shape[0]
        c.nnz = cl.shape[0]
        c.val_dtype = L.LYAP_F32 if vdt == np.float32 else L.LYAP_F64
        if inputs == "host":
            c.mem = L.LYAP_MEM_HOST
            arrs = (rp, cl, vl)
            c.rowptr, c.col, c.val = (a.ctypes.data for a in arrs)
        else:
            c.mem = L.LYAP_MEM_DEVICE
            t = self.torch
            arrs = (t.from_numpy(rp).to(self.device), t.from_numpy(cl).to(self.device), t.from_numpy(vl).to(self.device))
            c.rowptr, c.col, c.val = (a.data_ptr() for a in arrs)
        self._keep.append(arrs)
        return c

    def _make_rhs(self, C, inputs):
        C = np.ascontiguousarray(C, dtype=np.float64)
        if inputs == "host":
            self._keep.append(C)
            return C.ctypes.data
        t = self.torch.from_numpy(C).to(self.device)
        self._keep.append(t)
        return t.data_ptr()

    def solve(self) -> int:
        self.status = L.lyap_solve(self.h, self.stream)
        _, self.m, _ = L.lyap_residual_norm(self.h, 0)
        return self.status

    def history(self) -> np.ndarray:
        hist, m, _ = L.lyap_residual_norm(self.h, self.maxit)
        return hist[:m]

    def factor(self, tcap=None, z_dtype=None, out="device"):
        """Returns Z (n1 x t) for Lyapunov, (Z1, Z2) for Sylvester, as torch tensors (or numpy for out='host')."""
        t = self.torch
        if tcap is None:
            tcap = max(1, self.s * self.m)
        if z_dtype is None:
            z_dtype = "f32" if self.precision == L.LYAP_PREC_MIXED else "f64"
        zd = L.LYAP_F32 if z_dtype == "f32" else L.LYAP_F64
        dt = t.float32 if zd == L.LYAP_F32 else t.float64
        if out == "host":
            npdt = np.float32 if zd == L.LYAP_F32 else np.float64
            Z1 = np.zeros((self.n1, tcap), dtype=npdt)
            Z2 = np.zeros((self.n2, tcap), dtype=npdt) if self.sylv else None
            p1, p2 = Z1.ctypes.data, (Z2.ctypes.data if Z2 is not None else None)
            mem = L.LYAP_MEM_HOST
        else:
            Z1 = t.zeros((self.n1, tcap), dtype=dt, device=self.device)
            Z2 = t.zeros((self.n2, tcap), dtype=dt, device=self.device) if self.sylv else None
            p1, p2 = Z1.data_ptr(), (Z2.data_ptr() if Z2 is not None else None)
            mem = L.LYAP_MEM_DEVICE
        tk = L.lyap_factor(self.h, p1, tcap, p2, tcap, zd, mem, tcap, self.stream)
        Z1 = Z1[:, :tk]
        if self.sylv:
            return Z1, Z2[:, :tk]
        return Z1

    def projected(self, m: int, op: int = 0):
        """(ab, gamma, tau_next) of T_m (op 0) or J_m (op 1) from the device log."""
        return L.lyap_projected_matrix(self.h, op, m, self.s)

    def phase_times(self):
        return L.lyap_phase_times(self.h)

    def close(self):
        if getattr(self, "h", None):
            L.lyap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many Lyapunov equations solved together through lyap_batch_create/solve/factor.

    ``problems`` is a list of (A, C) with scipy CSR A and n x s C; all share ``maxit`` and
    ``precision``; ``tol`` is a scalar or one value per instance.
    """

    def __init__(self, problems, *, tol=1e-8, maxit=1000, precision="mixed", check_batch=32, pass2_blocks=16,
                 inputs="device", device="cuda:0", val_dtype="f32", check_every=1):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.count = len(problems)
        self.maxit = int(maxit)
        self.precision = PRECISIONS[precision]
        opt = L.lyap_default_options()
        opt.maxit = self.maxit
        opt.precision = self.precision
        opt.check_batch = int(check_batch)
        opt.pass2_blocks = int(pass2_blocks)
        opt.check_every = L.LYAP_CHECK_ADAPTIVE if check_every == "adaptive" else int(check_every)
        self.opt = opt
        self.s = [int(C.shape[1]) for _, C in problems]
        self.n = [int(A.shape[0]) for A, _ in problems]
        tols = list(tol) if hasattr(tol, "__len__") else [float(tol)] * self.count
        vdt = np.float32 if val_dtype == "f32" else np.float64
        self._keep = []
        helper = Solver.__new__(Solver)
        helper.torch, helper.device, helper._keep = torch, self.device, self._keep
        csrs = [Solver._make_csr(helper, A, inputs, vdt) for A, _ in problems]
        cptrs = [Solver._make_rhs(helper, C, inputs) for _, C in problems]
        self.ws_bytes = L.lyap_batch_workspace_size(csrs, self.s, opt)
        with torch.cuda.device(self.device):
            self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device).cuda_stream
        c_mem = L.LYAP_MEM_HOST if inputs == "host" else L.LYAP_MEM_DEVICE
        self.h = L.lyap_batch_create(csrs, cptrs, c_mem, self.s, tols, opt, self.ws.data_ptr(), self.ws_bytes,
                                     self.stream)
        self._keep.clear()

    def solve(self, autotune=False) -> int:
        return L.lyap_batch_solve(self.h, autotune, self.stream)

    def status(self):
        return L.lyap_batch_status(self.h, self.count)

    def history(self, i):
        return L.lyap_batch_residual_norm(self.h, i, self.maxit)[0]

    def factor(self, i, tcap=None, z_dtype=None):
        t = self.torch
        if tcap is None:
            tcap = max(1, self.s[i] * self.status()[1][i])
        if z_dtype is None:
            z_dtype = "f32" if self.precision == L.LYAP_PREC_MIXED else "f64"
        zd = L.LYAP_F32 if z_dtype == "f32" else L.LYAP_F64
        Z = t.zeros((self.n[i], tcap), dtype=t.float32 if zd == L.LYAP_F32 else t.float64, device=self.device)
        tk = L.lyap_batch_factor(self.h, i, Z.data_ptr(), tcap, zd, tcap, self.stream)
        return Z[:, :tk]

    def tuning(self):
        return L.lyap_batch_tuning(self.h)

    def phase_times(self):
        return L.lyap_batch_phase_times(self.h)

    def close(self):
        if getattr(self, "h", None):
            L.lyap_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ExtendedKrylov:
    """Extended Krylov projection (lyap_ek_*): inner solves by conjugate gradients preconditioned by
    Jacobi scaling, IC(0) applied by a truncated Neumann series, or the learned factor values, on
    the nx x ny grid ``grid`` (x fastest) of a 5-point operator."""

    PRECOND = {"jacobi": 0, "ic0": 1, "learned": 2}

    def __init__(self, A, C, *, tol=1e-8, maxit=60, inner_tol=1e-10, grid=None, device="cuda:0"):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.n = int(A.shape[0])
        self.s = int(C.shape[1])
        self.maxit = int(maxit)
        rp, cl, vl = csr_arrays(A)
        self._arrs = [torch.from_numpy(x).to(self.device) for x in (rp, cl, vl)]
        c = L.lyap_csr()
        c.n, c.nnz = self.n, cl.shape[0]
        c.rowptr, c.col, c.val = (a.data_ptr() for a in self._arrs)
        c.val_dtype, c.mem = L.LYAP_F64, L.LYAP_MEM_DEVICE
        nx, ny = grid if grid is not None else (0, 0)
        self.grid = (int(nx), int(ny))
        self.ws_bytes = L.lyap_ek_workspace_size(c, self.s, self.maxit, nx, ny)
        with torch.cuda.device(self.device):
            self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device).cuda_stream
        self._C = torch.from_numpy(np.ascontiguousarray(C, dtype=np.float64)).to(self.device)
        self.h = L.lyap_ek_create(c, self._C.data_ptr(), L.LYAP_MEM_DEVICE, self.s, tol, self.maxit, inner_tol, nx, ny,
                                  self.ws.data_ptr(), self.ws_bytes, self.stream)
        self.m = 0

    def precond_status(self) -> int:
        """0 when IC(0) exists on the grid (the IC(0) and learned preconditioners are available)."""
        return L.lyap_ek_precond_status(self.h)

    def solve(self, precond="jacobi", train_solves=1, train_iters=150, lr=3e-3) -> int:
        st = L.lyap_ek_solve(self.h, self.PRECOND[precond], train_solves, train_iters, lr, self.stream)
        _, self.m = L.lyap_ek_residual_norm(self.h, 0)
        return st

    def history(self):
        return L.lyap_ek_residual_norm(self.h, self.maxit)[0]

    def factor(self, tcap=None):
        t = self.torch
        if tcap is None:
            tcap = max(1, 2 * self.s * self.m)
        Z = t.zeros((self.n, tcap), dtype=t.float64, device=self.device)
        tk = L.lyap_ek_factor(self.h, Z.data_ptr(), tcap, tcap, self.stream)
        return Z[:, :tk]

    def stats(self):
        v = L.lyap_ek_stats(self.h, 7 + 2 * (self.maxit + 1))
        ns = int(v[4])
        its = [int(x) for x in v[7:7 + ns]]
        kinds = [int(x) for x in v[7 + ns:7 + 2 * ns]]
        return {"solve_ms": v[0], "train_ms": v[1], "loss_before": v[2], "loss_after": v[3], "fallbacks": int(v[5]),
                "network_accepted": bool(v[6]), "inner_iterations": its, "inner_kinds": kinds}

    def _cols(self, Bm):
        t = self.torch
        return t.from_numpy(np.asfortranarray(Bm, dtype=np.float64).T.copy()).to(self.device)  # K x n: column k contiguous

    def net_grad(self, params, B, X):
        """Energy loss and gradient of the network with parameters ``params`` over the pairs
        A X = B (n x K each, K <= 4)."""
        Bd, Xd = self._cols(B), self._cols(X)
        return L.lyap_ek_net_grad(self.h, params, B.shape[1], Bd.data_ptr(), Xd.data_ptr(), self.stream)

    def precond_apply(self, kind, R, params=None):
        """P R on the device (kind "ic0" or "learned"; the learned values from ``params`` when given)."""
        Rd = self._cols(R)
        Zd = self.torch.empty_like(Rd)
        L.lyap_ek_precond_apply(self.h, self.PRECOND[kind], params, R.shape[1], Rd.data_ptr(), Zd.data_ptr(), self.stream)
        self.torch.cuda.synchronize(self.device)
        return Zd.cpu().numpy().T.copy()

    def precond_values(self, kind):
        return L.lyap_ek_precond_values(self.h, self.PRECOND[kind], self.n)

    def close(self):
        if getattr(self, "h", None):
            L.lyap_ek_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Generalized:
    """A X E + E X A + C C^T = 0 with E symmetric positive definite (lyap_gen_*): block Lanczos
    with an E-orthonormal stored basis; the solves with E by Jacobi-preconditioned CG."""

    def __init__(self, A, E, C, *, tol=1e-8, maxit=300, inner_tol=1e-13, device="cuda:0"):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.n = int(A.shape[0])
        self.s = int(C.shape[1])
        self.maxit = int(maxit)
        self._keep = []
        csr = []
        for M in (A, E):
            rp, cl, vl = csr_arrays(M)
            arrs = [torch.from_numpy(x).to(self.device) for x in (rp, cl, vl)]
            self._keep.append(arrs)
            c = L.lyap_csr()
            c.n, c.nnz = self.n, cl.shape[0]
            c.rowptr, c.col, c.val = (a.data_ptr() for a in arrs)
            c.val_dtype, c.mem = L.LYAP_F64, L.LYAP_MEM_DEVICE
            csr.append(c)
        self.ws_bytes = L.lyap_gen_workspace_size(csr[0], csr[1], self.s, self.maxit)
        with torch.cuda.device(self.device):
            self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device).cuda_stream
        self._C = torch.from_numpy(np.ascontiguousarray(C, dtype=np.float64)).to(self.device)
        self.h = L.lyap_gen_create(csr[0], csr[1], self._C.data_ptr(), L.LYAP_MEM_DEVICE, self.s, tol, self.maxit,
                                   inner_tol, self.ws.data_ptr(), self.ws_bytes, self.stream)
        self.m = 0

    def solve(self) -> int:
        st = L.lyap_gen_solve(self.h, self.stream)
        _, self.m = L.lyap_gen_residual_norm(self.h, 0)
        return st

    def history(self):
        return L.lyap_gen_residual_norm(self.h, self.maxit)[0]

    def factor(self, tcap=None):
        t = self.torch
        if tcap is None:
            tcap = max(1, self.s * self.m)
        Z = t.zeros((self.n, tcap), dtype=t.float64, device=self.device)
        tk = L.lyap_gen_factor(self.h, Z.data_ptr(), tcap, tcap, self.stream)
        return Z[:, :tk]

    def stats(self):
        v = L.lyap_gen_stats(self.h)
        return {"solve_ms": v[0], "e_solves": int(v[1]), "cg_iterations": int(v[2]), "cg_max": int(v[3])}

    def close(self):
        if getattr(self, "h", None):
            L.lyap_gen_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
