"""Write tests/golden/oracle_solves.json from the CPU oracle only.

For each named workload: the oracle's PCG iteration count to the workload's
tolerance (Fletcher-Reeves CG, V(2,2) Chebyshev(2)-Jacobi cycle, defaults of
the library), its final recurrence and true relative residuals, and the 2-norm
of the solution.  The benchmark's CPU-baseline and reference legs use the
iteration count to turn a bounded sample of oracle iterations into DOF/s to
tolerance.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import mg_inputs as mi  # noqa: E402
import oracle  # noqa: E402


def main():
    out = {}
    for name in ("poisson33_fp64", "adjoint129", "poisson257_c1e4"):
        dims, k, f, spec = mi.workload(name)
        O = oracle.Oracle(k)
        t = time.time()
        x, it, info = O.pcg(f, spec["rtol"], maxit=3000)
        out[name] = dict(dims=list(dims), rtol=spec["rtol"], iterations=it, rel_resid=info["rel_resid"],
                         true_rel_resid=info["true_rel_resid"], x_norm2=float(np.linalg.norm(x)),
                         oracle_seconds=round(time.time() - t, 2))
        print(name, out[name], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_solves.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
