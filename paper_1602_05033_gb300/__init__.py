"""GB300 projection solver for large symmetric Lyapunov and Sylvester equations.

Palitta & Simoncini, "Computationally enhanced projection methods for symmetric
Sylvester and Lyapunov matrix equations": block Lanczos with CholQR2
normalisation (Alg. 2), the cheap residual norm from the eigenpairs of the
projected block-tridiagonal matrix (Prop. 3.1, Alg. 3/4), and the two-pass
low-rank factor (Sec. 3.3).

The compute path is liblyap.so (hand-written CUDA for sm_103a behind the C ABI
of include/lyap.h).  ``_lib`` binds that ABI one-to-one; ``Solver`` is a thin
convenience layer that allocates the workspace and the factor with PyTorch.
"""
from ._lib import (  # noqa: F401
    LYAP_F32,
    LYAP_F64,
    LYAP_MEM_DEVICE,
    LYAP_MEM_HOST,
    LYAP_PREC_F64,
    LYAP_PREC_MIXED,
    LyapError,
    lyap_create,
    lyap_default_options,
    lyap_destroy,
    lyap_factor,
    lyap_phase_times,
    lyap_projected_matrix,
    lyap_residual_norm,
    lyap_solve,
    lyap_workspace_size,
    status_string,
)
from .solver import Batch, ExtendedKrylov, Generalized, Solver, csr_arrays  # noqa: F401
