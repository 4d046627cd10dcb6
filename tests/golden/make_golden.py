"""Write the stored expected values under tests/golden/ from the CPU oracle only.

oracle_solves.json: for each named workload, the oracle's PCG iteration count
to the workload's tolerance (Fletcher-Reeves CG, V(2,2) Chebyshev(2)-Jacobi
cycle, defaults of the library), its final recurrence and true relative
residuals, and the 2-norm of the solution.

oracle_spread.json (--spread): how far rounding order alone moves the oracle's
solves.  Each case is solved twice by the oracle, once with its default
summation order (sequential dot products, operator rows in increasing column
order) and once with the second fixed order (pairwise dot products, rows in
decreasing column order); the file records both iteration counts, the
relative 2-norm distance of the two solutions at tolerance and after the same
number of iterations.  These spreads are the evidence behind the tolerances
of the GPU solve-parity tests.

Run: python tests/golden/make_golden.py [--spread]
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

HERE = os.path.dirname(os.path.abspath(__file__))


def solves():
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
    with open(os.path.join(HERE, "oracle_solves.json"), "w") as fh:
        json.dump(out, fh, indent=1)


# (case name, workload name or None, grid N override, explicit (dims, block, lo, hi, seed), rtol, oracle kwargs)
SPREAD_CASES = [
    ("poisson33_fp64", "poisson33_fp64", None, None, None, {}),
    ("adjoint129", "adjoint129", None, None, None, {}),
    ("poisson257_c1e4_at65", "poisson257_c1e4", 65, None, None, {}),
    ("galerkin65_c1e6", None, None, ((65, 65, 65), 8, -3.0, 3.0, 78), 1e-10, dict(galerkin=True)),
    ("poisson257_c1e4", "poisson257_c1e4", None, None, None, {}),
]


def spread():
    out = {}
    for name, wl, n, explicit, rtol, kw in SPREAD_CASES:
        if wl is not None:
            dims, k, f, spec = mi.workload(wl, n)
            rtol = spec["rtol"]
        else:
            dims, block, lo, hi, seed = explicit
            k = mi.cell_k(dims, block, lo, hi, seed)
            f = mi.rhs_f(dims, seed)
        t = time.time()
        O0 = oracle.Oracle(k, **kw)
        O1 = oracle.Oracle(k, sum_order=1, **kw)
        x0, i0, _ = O0.pcg(f, rtol, maxit=3000)
        x1, i1, _ = O1.pcg(f, rtol, maxit=3000)
        m = min(i0, i1)
        xa, _, _ = O0.pcg(f, 0.0, maxit=m)
        xb, _, _ = O1.pcg(f, 0.0, maxit=m)
        nrm = np.linalg.norm(x0)
        out[name] = dict(dims=list(dims), rtol=rtol, options={k_: v_ for k_, v_ in kw.items()},
                         iterations_sequential=i0, iterations_pairwise=i1,
                         rel2_at_tolerance=float(np.linalg.norm(x1 - x0) / nrm),
                         rel2_at_equal_iterations=float(np.linalg.norm(xb - xa) / np.linalg.norm(xa)),
                         equal_iterations=m, oracle_seconds=round(time.time() - t, 1))
        print(name, out[name], flush=True)
    with open(os.path.join(HERE, "oracle_spread.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    if "--spread" in sys.argv:
        spread()
    else:
        solves()
