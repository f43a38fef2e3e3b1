"""Plain FP64 CPU oracle for the projection method of Palitta & Simoncini.

TEST INFRASTRUCTURE ONLY.  This package is a deliberately slow, direct
restatement of the paper's algorithms in NumPy/SciPy, used to check the CUDA
path.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the library itself never calls it and has no CPU
fallback.  It shares no code with the CUDA path: the only common module is
``workloads`` (seeded problem generators, which hold none of the method).

Modules
-------
lyap       block Lanczos (Alg. 2), cheap residual (Prop. 3.1 / Alg. 3),
           truncated factor (eq. 2.5, Sec. 3.2) and the two-pass device (Sec. 3.3)
sylvester  two-sided variant for A X + X B + C1 C2^T = 0 (Sec. 5.1, Alg. 4)
sylvester_small  A large and B small: only A projected, B diagonalised once (Sec. 5.2, Alg. 5)
lyap_general     A X E + E X A + C C^T = 0 with E symmetric positive definite, by Cholesky of E
explicit   explicit residual norms used as pins (dense and exact low-rank form)
ek         extended Krylov space K_m(A, C) + K_m(A^{-1}, A^{-1} C) with exact inner solves (Sec. 4)
cnn        convolutional preconditioner of the inner solves: forward, gradients, losses
pcg        inner solves with A by conjugate gradients: Jacobi, IC(0) and MIC(0) preconditioning
learned_factor   a network predicting the IC(0)-pattern factor values: loss, gradients
neumann_ic       IC(0) applied by a truncated Neumann series (products only), and the network-corrected
                 factor values trained with the energy-norm loss on solve pairs: loss, gradients, Adam
"""
from . import lyap, sylvester, explicit  # noqa: F401
