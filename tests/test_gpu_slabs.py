"""The z-slab domain decomposition of the solve (mg_params.slabs), through the
C ABI, against the oracle and against the single-domain GPU solve.

A decomposed solve runs the same kernels on every slab, with each stencil and
transfer pass reading its neighbours' boundary planes from halo planes filled
by an exchange, every dot product summed per slab and then over the slabs,
and the agglomeration level handed to the whole-grid hierarchy (its bottom
kernel) and back.  Only the summation order of the dot products differs from
the single-domain solve, so it meets the same float64 parity bar against the
oracle (both summation orders, equal iteration counts) and follows the
single-domain solve to rounding.
"""
import numpy as np
import pytest
import torch

import mg_inputs as mi
import oracle
from oracle_orders import check_fp64_solve_against_both_oracle_orders

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def N(t):
    return t.detach().cpu().numpy()


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("slabs", [2, 3, 4])
@pytest.mark.parametrize("name,n", [("poisson33_fp64", None), ("poisson257_c1e4", 65)])
def test_slab_solve_fp64_matches_oracle(gpu_lib, name, n, slabs):
    mg = gpu_lib
    dims, k, f, spec = mi.workload(name, n)
    S = mg.MGSolver(T(k), mg.Params(maxit=2000, slabs=slabs))
    x, st = S.solve(T(f), spec["rtol"])
    assert st.true_rel_resid <= spec["rtol"] * 1.01
    check_fp64_solve_against_both_oracle_orders(N(x), st.iters, st.history, f, k, spec["rtol"],
                                                hist_its=10 if name == "poisson257_c1e4" else None)


@pytest.mark.parametrize("params", [dict(), dict(precision="mixed_fp32"), dict(precision="mixed_bf16k"),
                                    dict(coarse_op="galerkin"), dict(coarse_op="galerkin", precision="mixed_fp32"),
                                    dict(smoother="richardson", nu_pre=8, nu_post=8), dict(cheby_degree=3),
                                    dict(stencil_kernel=2), dict(flexible=1), dict(slab_level=1),
                                    dict(nu_pre=0, nu_post=2)])
def test_slab_solve_follows_the_single_domain_solve(gpu_lib, params):
    """Every precision, coarse operator, smoother, kernel choice and
    agglomeration level: the decomposed solve (3 slabs) takes the
    single-domain solve's iterations and reaches the same solution to
    rounding (only the dot products' summation order differs)."""
    mg = gpu_lib
    dims = (65, 65, 65)
    k = mi.cell_k(dims, 8, -1.5, 1.5, 91)
    f = mi.rhs_f(dims, 91)
    x1, st1 = mg.MGSolver(T(k), mg.Params(maxit=500, **params)).solve(T(f), 1e-10)
    x3, st3 = mg.MGSolver(T(k), mg.Params(maxit=500, slabs=3, **params)).solve(T(f), 1e-10)
    assert st3.status == "MG_OK" and abs(st3.iters - st1.iters) <= 1, (st1.iters, st3.iters)
    assert st3.true_rel_resid <= 1.05e-10
    assert rel2(N(x3), N(x1)) < 1e-9


def test_slab_galerkin_high_contrast_matches_oracle(gpu_lib):
    """Galerkin coarse operators at contrast 10^6, 4 slabs: the float64
    parity bar against the oracle's Galerkin hierarchy."""
    mg = gpu_lib
    dims = (65, 65, 65)
    k = mi.cell_k(dims, 8, -3.0, 3.0, 78)
    f = mi.rhs_f(dims, 78)
    x, st = mg.MGSolver(T(k), mg.Params(maxit=400, coarse_op="galerkin", slabs=4)).solve(T(f), 1e-10)
    check_fp64_solve_against_both_oracle_orders(N(x), st.iters, st.history, f, k, 1e-10,
                                                oracle_kw=dict(galerkin=True), hist_its=20)


@pytest.mark.parametrize("dims,slabs", [((33, 17, 65), 2), ((33, 33, 9), 3), ((65, 17, 33), 7)])
def test_slab_solve_non_cubic_and_uneven(gpu_lib, dims, slabs):
    """Non-cubic grids and uneven splits (the agglomeration level's planes do
    not divide by the slab count; 7 slabs of 2-3 coarse planes).  A wrong halo
    would change the operator or the preconditioner from the first iteration:
    ten iterations are compared iterate by iterate with the oracle, and the
    oracle's operator confirms the true residual of the converged solution.
    (These anisotropic problems converge slowly, about 5% per iteration near
    the tolerance, so rounding alone moves the stopping iteration by a few
    of their ~170.)"""
    mg = gpu_lib
    k = mi.cell_k(dims, 2, -2.0, 2.0, 92)
    f = mi.rhs_f(dims, 92)
    O = oracle.Oracle(k)
    x10o, _, _ = O.pcg(f, 0.0, maxit=10)
    x10, st10 = mg.MGSolver(T(k), mg.Params(maxit=10, slabs=slabs)).solve(T(f), 0.0, raise_on_error=False)
    assert st10.iters == 10 and rel2(N(x10), x10o) < 1e-10
    _, ito, _ = O.pcg(f, 1e-10, maxit=500)
    x, st = mg.MGSolver(T(k), mg.Params(maxit=500, slabs=slabs)).solve(T(f), 1e-10)
    true = np.linalg.norm((f - O.apply(N(x)))[1:-1, 1:-1, 1:-1]) / np.linalg.norm(f)
    assert true <= 1.01e-10
    assert abs(st.iters - ito) <= max(1, ito // 30)


def test_slab_solve_host_buffers_and_repeatability(gpu_lib):
    mg = gpu_lib
    dims, k, f, spec = mi.workload("poisson33_fp64", 65)
    S = mg.MGSolver(T(k), mg.Params(slabs=4, precision="mixed_fp32"))
    a, s1 = S.solve(T(f), 1e-10)
    b, s2 = S.solve(T(f), 1e-10)
    assert s1.iters == s2.iters and torch.equal(a, b)
    xh = torch.zeros(dims, dtype=torch.float64)
    sh = S.solve_host(torch.tensor(f), xh, 1e-10)
    assert sh.iters == s1.iters and torch.equal(xh, a.cpu())


def test_slab_adjoint_gradient_matches_single_domain(gpu_lib):
    mg = gpu_lib
    dims = (33, 33, 33)
    k = mi.cell_k(dims, 4, -1.0, 1.0, 93)
    f = mi.rhs_f(dims, 93)
    mask = T(mi.obs_mask(dims, 93).astype(np.float64))
    grads = []
    for slabs in (1, 2):
        logk = T(np.log(k)).requires_grad_(True)
        phi = mg.mg_solve(T(f), logk, mg.Params(slabs=slabs), rtol=1e-12)
        (0.5 * (phi ** 2 * mask).sum()).backward()
        grads.append(N(logk.grad))
    assert rel2(grads[1], grads[0]) < 1e-8


def test_slab_parameters_rejected(gpu_lib):
    mg = gpu_lib
    dims, k, f, spec = mi.workload("poisson33_fp64")
    for params in (dict(slabs=2, krylov="fgmres"), dict(slabs=2, stencil_kernel=1), dict(slabs=2, nonzero_guess=1),
                   dict(slabs=16), dict(slabs=0), dict(slabs=65)):
        with pytest.raises(mg.MgError) as e:
            mg.MGSolver(T(k), mg.Params(**params))
        assert e.value.status == "MG_ERR_ARG", params
