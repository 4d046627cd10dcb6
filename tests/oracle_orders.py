"""Comparison of a float64 GPU solve with the oracle's solves in both of the
oracle's summation orders (shared by the GPU parity tests)."""
import numpy as np

import oracle


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def check_fp64_solve_against_both_oracle_orders(xg, itg, hist, f, k, rtol, oracle_kw=None, hist_its=None):
    """The float64 GPU solve (solution xg after itg iterations) against the
    oracle's solves in both of its summation orders (sequential and pairwise:
    the method fixes none, so both are faithful).

    - The iteration count to rtol is within 1 of one of the orders.
    - The solutions are compared after the same number of iterations (the
      oracle is run for exactly itg iterations when its own count differs):
      two runs that stop one iteration apart differ by that iteration's
      update whatever their rounding, which is not a parity defect.  The GPU
      must then be within relative 1e-10 in the 2-norm of one order.  Where
      rounding order alone moves a high-contrast solve by more than that, the
      oracle's two orders measure by how much (their distance d): the GPU's
      sums are a third fixed order, so it must be no farther than d from the
      nearer oracle order and, by the triangle inequality, no farther than
      2 d from the other (each plus 1e-10).
    - The residual history follows the nearest order's over hist_its
      iterations (all when None).
    Returns (errors at equal iterations, oracle spread at equal iterations)."""
    kw = oracle_kw or {}
    its, hists, at_itg = [], [], []
    for order in (0, 1):
        O = oracle.Oracle(k, sum_order=order, **kw)
        xo, ito, info = O.pcg(f, rtol, maxit=3000)
        its.append(ito)
        hists.append(info["hist"])
        at_itg.append(xo if ito == itg else O.pcg(f, 0.0, maxit=itg)[0])
        del O
    assert min(abs(itg - i) for i in its) <= 1, (itg, its)
    spread = rel2(at_itg[1], at_itg[0])
    errs = [rel2(xg, x) for x in at_itg]
    assert min(errs) <= 1e-10 or (min(errs) <= spread + 1e-10 and max(errs) <= 2 * spread + 1e-10), (
        itg, its, errs, spread)
    ho = hists[0] if abs(itg - its[0]) <= abs(itg - its[1]) else hists[1]
    h = np.asarray(hist)
    m = min(len(h), len(ho), hist_its or len(h))
    assert np.max(np.abs(h[:m] - ho[:m]) / ho[:m]) < 1e-6
    return errs, spread
