"""Iteration count of the method on the benchmark workload, from the oracle.

Runs the FP64 oracle's SAP-FGMRES(16) to a relative residual of 1e-10 on the
16^3x32 workload (eps 0.5, c_sw 1.0, kappa 0.125, 8x4x4x4 domains, nmr 4,
ncy 4, Gaussian source) and writes the counts to iterations_16c32.json.  A
GPU test holds the CUDA path's solve of the same workload to this iteration
count (within one) and residual history.  Only oracle/ code runs here.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import pyoracle as ora  # noqa: E402
from paper_1502_04025_gb300 import inputs  # noqa: E402

WORKLOAD = dict(L=(16, 16, 16, 32), dom=(8, 4, 4, 4), eps=0.5, csw=1.0, kappa=0.125, gauge_seed=1002,
                source_seed=2002, nmr=4, ncy=4, m=16, tol=1e-10)


def main():
    w = WORKLOAD
    U = inputs.gauge_field(w["L"], w["eps"], w["gauge_seed"])
    A = ora.clover(w["L"], U, w["csw"], w["kappa"])
    Ainv = ora.invert_clover(w["L"], A)
    b = inputs.gaussian_source(w["L"], w["source_seed"])
    t0 = time.time()
    x, info = ora.fgmres(w["L"], w["dom"], U, A, Ainv, w["kappa"], b, w["tol"], m=w["m"], max_restarts=50,
                         use_sap=True, nmr=w["nmr"], ncy=w["ncy"])
    out = dict(workload={k: list(v) if isinstance(v, tuple) else v for k, v in w.items()},
               iterations=info["iters"], restarts=info["restarts"], converged=info["converged"],
               true_rel_res=info["true_rel_res"], seconds=time.time() - t0,
               history=[float(h) for h in info["history"]])
    with open(os.path.join(HERE, "iterations_16c32.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("iterations", "restarts", "converged", "true_rel_res", "seconds")}))


if __name__ == "__main__":
    main()
