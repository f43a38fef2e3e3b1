"""Writes oracle-computed reference values for the full-size workloads.

Calls only oracle/ and workloads/ (never the CUDA path).  The n = 1e6 history
takes about a minute of CPU time, too long to recompute inside the test suite,
so it is stored here:

    python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402
from oracle import explicit, lyap  # noqa: E402


def main():
    P = wl.config_c2(0)
    t0 = time.time()
    res = lyap.solve(P.A, P.C1, tol=P.tol, maxit=P.maxit)
    secs = time.time() - t0
    # truncation threshold of eq. 2.5 tied to tol (oracle.lyap.auto_trunc_eps)
    M, sig = lyap.truncated_factor(res.log, res.m, None, P.tol)
    Z, _ = lyap.factor(P.A, P.C1, res)
    true_rel = explicit.lyap_lowrank(P.A, Z, P.C1) / res.log.beta**2
    out = {
        "workload": "Lyapunov, 3D 7-point Laplacian on 100^3 (n = 1e6), s = 4, C = rhs(n, 4, seed=0), tol 1e-8, maxit 400",
        "source": "oracle.lyap.solve / truncated_factor (FP64 NumPy/SciPy), tests/golden/make_oracle_golden.py",
        "m": int(res.m),
        "converged": bool(res.converged),
        "history": [float(x) for x in res.history],
        "beta": float(res.log.beta),
        "t": int(M.shape[1]),
        "sigma": [float(x) for x in sig],
        "explicit_rel_residual": float(true_rel),
        "oracle_seconds_on_generating_host": secs,
        "generating_host_cores": os.cpu_count(),
    }
    with open(os.path.join(HERE, "oracle_c2_lap3d100_s4.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("m", res.m, "t", M.shape[1], "explicit", true_rel, "secs", round(secs, 1))


if __name__ == "__main__":
    main()
