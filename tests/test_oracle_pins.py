"""Pins for the CPU oracle: checks against closed forms, invariants, library
routines and brute force, independent of the oracle's own code.

Each test names the property of the paper's method (or of the mathematics)
that fixes the expected value.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import mg_inputs as mi
import oracle

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def grid(dims):
    """Node coordinates (z, y, x) of a unit-cube vertex grid."""
    nz, ny, nx = dims
    z = np.linspace(0, 1, nz)[:, None, None]
    y = np.linspace(0, 1, ny)[None, :, None]
    x = np.linspace(0, 1, nx)[None, None, :]
    return z, y, x


def interior(a):
    return a[1:-1, 1:-1, 1:-1]


def dense_A(O, l=0):
    rp, col, val = O.csr(l)
    n = len(rp) - 1
    return sp.csr_matrix((val, col, rp), shape=(n, n))


# ------------------------------------------------------------------ operator
def test_default_levels_match_hierarchy_depth():
    # 33^3 -> 4 levels ending at 3^3 interior; 257^3 -> 7; 513^3 -> 8; 1025^3 -> 9
    assert oracle.default_levels((33,) * 3) == 4
    assert oracle.default_levels((129,) * 3) == 6
    assert oracle.default_levels((257,) * 3) == 7
    assert oracle.default_levels((513,) * 3) == 8
    assert oracle.default_levels((1025,) * 3) == 9
    assert oracle.default_levels((9, 17, 33)) == 2


@pytest.mark.parametrize("dims", [(9, 17, 33), (17, 9, 5)])
def test_constant_k_sine_eigenpairs(dims):
    """k = 1: sin modes are eigenvectors with lambda = sum_a 4/h_a^2 sin^2(m_a pi h_a / 2)."""
    O = oracle.Oracle(np.ones(tuple(d - 1 for d in dims)), levels=1)
    z, y, x = grid(dims)
    h = [1.0 / (d - 1) for d in dims]
    for m in [(1, 1, 1), (2, 3, 1), (3, 1, 2)]:
        v = np.sin(m[0] * np.pi * z) * np.sin(m[1] * np.pi * y) * np.sin(m[2] * np.pi * x)
        lam = sum(4.0 / ha ** 2 * np.sin(ma * np.pi * ha / 2) ** 2 for ma, ha in zip(m, h))
        Av = O.apply(v)
        assert np.max(np.abs(interior(Av) - lam * interior(v))) <= 1e-11 * lam


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("face_rule", [0, 1])
def test_layered_k_closed_form(axis, face_rule):
    """k constant on layers normal to one axis: the edge coefficients parallel to
    the layers are the two-layer mean (harmonic or arithmetic), those normal to
    them are the layer value, so A acting on sin*sin*w separates into a known
    tridiagonal expression along the layered axis."""
    dims = [11, 9, 13]
    nl = dims[axis] - 1
    rng = np.random.default_rng(3)
    kap = 10.0 ** rng.uniform(-2, 2, nl)
    shape = [d - 1 for d in dims]
    k = np.broadcast_to(kap.reshape([nl if a == axis else 1 for a in range(3)]), shape).copy()
    O = oracle.Oracle(k, levels=1, face_rule=face_rule)
    coords = grid(dims)
    h = [1.0 / (d - 1) for d in dims]
    others = [a for a in range(3) if a != axis]
    m = {others[0]: 2, others[1]: 1}
    u = np.ones(dims)
    for a in others:
        u = u * np.sin(m[a] * np.pi * coords[a])
    w = np.zeros(dims[axis])
    w[1:-1] = rng.uniform(-1, 1, dims[axis] - 2)
    u = u * w.reshape([-1 if a == axis else 1 for a in range(3)])
    Au = O.apply(u)
    # expected value at node with layered index K: s * [mean_K * w_K * sum_lam + tridiag]
    sum_lam = sum(4.0 / h[a] ** 2 * np.sin(m[a] * np.pi * h[a] / 2) ** 2 for a in others)
    K = np.arange(1, dims[axis] - 1)
    kl, kr = kap[K - 1], kap[K]
    mean = 2.0 / (1.0 / kl + 1.0 / kr) if face_rule == 0 else 0.5 * (kl + kr)
    tri = (kr * (w[K] - w[K + 1]) + kl * (w[K] - w[K - 1])) / h[axis] ** 2
    line = np.zeros(dims[axis])
    line[K] = mean * w[K] * sum_lam + tri
    s = np.ones(dims)
    for a in others:
        s = s * np.sin(m[a] * np.pi * coords[a])
    expect = s * line.reshape([-1 if a == axis else 1 for a in range(3)])
    scale = np.max(np.abs(expect))
    assert np.max(np.abs(interior(Au) - interior(expect))) <= 1e-12 * scale


def _manufactured(N, face_rule, smooth_k):
    dims = (N,) * 3
    z, y, x = grid(dims)
    phi = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    if smooth_k:
        hc = 1.0 / (N - 1)
        zc = (np.arange(N - 1) + 0.5)[:, None, None] * hc
        yc = (np.arange(N - 1) + 0.5)[None, :, None] * hc
        xc = (np.arange(N - 1) + 0.5)[None, None, :] * hc
        kc = np.exp(xc + 0.5 * yc - 0.3 * zc)
        kn = np.exp(x + 0.5 * y - 0.3 * z)
        px = np.pi * np.cos(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        py = np.pi * np.sin(np.pi * x) * np.cos(np.pi * y) * np.sin(np.pi * z)
        pz = np.pi * np.sin(np.pi * x) * np.sin(np.pi * y) * np.cos(np.pi * z)
        f = kn * (3 * np.pi ** 2 * phi - (1.0 * px + 0.5 * py - 0.3 * pz))
    else:
        kc = np.ones((N - 1,) * 3)
        f = 3 * np.pi ** 2 * phi
    f[0, :, :] = f[-1, :, :] = f[:, 0, :] = f[:, -1, :] = f[:, :, 0] = f[:, :, -1] = 0
    O = oracle.Oracle(kc, face_rule=face_rule)
    sol, it, info = O.pcg(f, 1e-12)
    assert info["true_rel_resid"] < 1e-11
    return np.max(np.abs(sol - phi))


@pytest.mark.parametrize("smooth_k,face_rule", [(False, 0), (True, 0), (True, 1)])
def test_manufactured_solution_second_order(smooth_k, face_rule):
    """-div(k grad phi) = f with phi = sin sin sin: the max-norm error of the
    discrete solution decays like h^2 (ratio 4 per halving) for constant k and
    for a smooth k sampled per cell; a mis-centred edge coefficient would
    drop the ratio towards 2."""
    errs = [_manufactured(N, face_rule, smooth_k) for N in (9, 17, 33, 65)]
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert 3.7 < ratios[-1] < 4.3, ratios
    assert 3.4 < ratios[-2] < 4.6, ratios


@pytest.mark.parametrize("face_rule", [0, 1])
def test_operator_symmetric_positive_and_rowsums(face_rule):
    dims = (9, 11, 13)
    k = mi.cell_k(dims, 2, -2, 2, seed=11)
    O = oracle.Oracle(k, levels=1, face_rule=face_rule)
    A = dense_A(O).toarray()
    assert np.max(np.abs(A - A.T)) <= 1e-13 * np.max(np.abs(A))
    assert np.min(np.linalg.eigvalsh(A)) > 0
    # A 1 = 0 on rows whose 6 neighbours are all interior
    one = np.zeros(dims)
    one[1:-1, 1:-1, 1:-1] = 1.0
    A1 = O.apply(one)
    deep = A1[2:-2, 2:-2, 2:-2]
    assert np.max(np.abs(deep)) <= 1e-12 * np.max(np.abs(A))
    # x^T A y = y^T A x and x^T A x > 0 through the matrix-free apply as well
    x = mi.random_nodal(dims, 1)
    yv = mi.random_nodal(dims, 2)
    assert abs(np.sum(x * O.apply(yv)) - np.sum(yv * O.apply(x))) <= 1e-12 * np.abs(A).max() * np.sum(x * x)
    assert np.sum(x * O.apply(x)) > 0


def test_jacobi_spectrum_bound():
    """Gershgorin: eigenvalues of D^-1 A lie in (0, 2] since diag = sum |offdiag| (+ boundary terms)."""
    dims = (9, 9, 9)
    k = mi.cell_k(dims, 2, -3, 3, seed=5)
    A = dense_A(oracle.Oracle(k, levels=1)).toarray()
    d = np.diag(A)
    ev = np.linalg.eigvalsh(A / np.sqrt(np.outer(d, d)))
    assert ev.min() > 0 and ev.max() <= 2.0 + 1e-12


@pytest.mark.parametrize("N", [5, 9])
def test_pcg_matches_dense_direct_solve(N):
    dims = (N,) * 3
    k = mi.cell_k(dims, 2, -1, 1, seed=7)
    f = mi.rhs_f(dims, 7)
    O = oracle.Oracle(k)
    x, it, info = O.pcg(f, 1e-14, maxit=200)
    A = dense_A(O).toarray()
    xd = np.linalg.solve(A, interior(f).ravel())
    assert np.max(np.abs(interior(x).ravel() - xd)) <= 1e-11 * np.max(np.abs(xd))
    assert np.all(x[0] == 0) and np.all(x[:, :, -1] == 0)


# ------------------------------------------------------------------ coarse k
def test_coarse_k_exact_for_aligned_blocks():
    """With block size B and 2^l <= B, all 8 children of a coarse cell share one
    block value, so every averaging rule returns that value."""
    dims = (33,) * 3
    B = 8
    lk = mi.cell_log10_k(dims, B, -1, 1, seed=1)
    for rule in (0, 1, 2):
        O = oracle.Oracle(10.0 ** lk, coarse_rule=rule)
        for l in range(1, O.levels):
            s = 2 ** l
            expect = 10.0 ** lk[::s, ::s, ::s]
            np.testing.assert_allclose(O.cells(l), expect, rtol=1e-14)


def test_coarse_k_rules_on_two_value_children():
    """Children {a (4 cells), b (4 cells)}: arithmetic (a+b)/2, geometric sqrt(ab),
    harmonic 2ab/(a+b)."""
    dims = (5, 5, 5)
    a, b = 3.0, 0.25
    k = np.full((4, 4, 4), a)
    k[:, :, 1::2] = b
    got = [oracle.Oracle(k, levels=2, coarse_rule=r).cells(1) for r in (0, 1, 2)]
    np.testing.assert_allclose(got[0], (a + b) / 2, rtol=1e-15)
    np.testing.assert_allclose(got[1], math.sqrt(a * b), rtol=1e-14)
    np.testing.assert_allclose(got[2], 2 * a * b / (a + b), rtol=1e-15)


# ------------------------------------------------------------------ smoother
@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_chebyshev_error_polynomial_on_eigenvectors(degree):
    """Constant k: D is a multiple of I and the sine modes are eigenvectors of
    D^-1 A with eigenvalue mu; one sweep multiplies the error in that mode by
    T_m((theta - mu)/delta) / T_m(theta/delta) (Chebyshev polynomial of the
    first kind, evaluated with numpy)."""
    dims = (17, 17, 17)
    lo_frac, hi = 0.1, 2.0
    O = oracle.Oracle(np.ones((16, 16, 16)), levels=1, degree=degree, eig_lo_frac=lo_frac, eig_hi=hi)
    alpha, beta = lo_frac * hi, hi
    theta, delta = (beta + alpha) / 2, (beta - alpha) / 2
    Tm = np.polynomial.chebyshev.Chebyshev.basis(degree)
    z, y, x = grid(dims)
    h = 1.0 / 16
    D = 6.0 / h ** 2
    for m in [(1, 1, 1), (5, 2, 7), (15, 15, 15)]:
        v = np.sin(m[0] * np.pi * z) * np.sin(m[1] * np.pi * y) * np.sin(m[2] * np.pi * x)
        mu = sum(4.0 / h ** 2 * np.sin(mm * np.pi * h / 2) ** 2 for mm in m) / D
        factor = Tm((theta - mu) / delta) / Tm(theta / delta)
        # error propagation from x0 = v with b = 0
        out = O.smooth(np.zeros(dims), v)
        assert np.max(np.abs(out - factor * v)) <= 1e-12
        # zero initial guess with exact solution v: x_m = (1 - factor) v
        out0 = O.smooth(O.apply(v))
        assert np.max(np.abs(out0 - (1 - factor) * v)) <= 1e-12


@pytest.mark.parametrize("omega", [1.0, 6.0 / 7.0, 0.5])
def test_richardson_jacobi_error_factor_on_eigenvectors(omega):
    """Richardson preconditioned with Jacobi, x += omega D^-1 (b - A x): on a
    constant-k sine mode with D^-1 A eigenvalue mu one iteration multiplies the
    error by 1 - omega mu; from a zero guess it returns omega D^-1 b."""
    dims = (17, 17, 17)
    O = oracle.Oracle(np.ones((16, 16, 16)), levels=1, smoother=1, omega=omega)
    z, y, x = grid(dims)
    h = 1.0 / 16
    D = 6.0 / h ** 2
    for m in [(1, 1, 1), (5, 2, 7), (15, 15, 15)]:
        v = np.sin(m[0] * np.pi * z) * np.sin(m[1] * np.pi * y) * np.sin(m[2] * np.pi * x)
        mu = sum(4.0 / h ** 2 * np.sin(mm * np.pi * h / 2) ** 2 for mm in m) / D
        out = O.smooth(np.zeros(dims), v)
        assert np.max(np.abs(out - (1 - omega * mu) * v)) <= 1e-12
        out0 = O.smooth(O.apply(v))
        assert np.max(np.abs(out0 - omega * mu * v)) <= 1e-12


def test_richardson_vcycle_symmetric_positive_definite_and_mesh_independent():
    """With the same Richardson iterations before and after the correction the
    V-cycle is symmetric; with omega D^-1 A of spectral radius below 2 it is
    positive definite, so CG applies, and (with 8 iterations per level, as in
    Sec. 5) the CG iteration count does not grow with the mesh."""
    dims = (17, 17, 17)
    k = mi.cell_k(dims, 4, -1, 1, seed=9)
    O = oracle.Oracle(k, nu_pre=8, nu_post=8, smoother=1, omega=6.0 / 7.0)
    x = mi.random_nodal(dims, 1)
    y = mi.random_nodal(dims, 2)
    Mx, My = O.vcycle(x), O.vcycle(y)
    assert abs(np.sum(Mx * y) - np.sum(x * My)) <= 1e-13 * np.sqrt(np.sum(Mx ** 2) * np.sum(y ** 2))
    assert np.sum(Mx * x) > 0 and np.sum(My * y) > 0
    its = []
    for N in (9, 17, 33, 65):
        d = (N,) * 3
        On = oracle.Oracle(np.ones((N - 1,) * 3), nu_pre=8, nu_post=8, smoother=1, omega=6.0 / 7.0)
        _, it, _ = On.pcg(mi.rhs_f(d, 3), 1e-8)
        its.append(it)
    assert max(its) - min(its) <= 2, its


def test_chebyshev_degree_10_vcycle_symmetric_and_mesh_independent():
    """Chebyshev(10)-Jacobi, the smoother of the paper's RASM comparison (Sec. 5)."""
    its = []
    for N in (9, 17, 33, 65):
        d = (N,) * 3
        On = oracle.Oracle(np.ones((N - 1,) * 3), degree=10)
        _, it, _ = On.pcg(mi.rhs_f(d, 3), 1e-8)
        its.append(it)
    assert max(its) - min(its) <= 2, its
    dims = (17, 17, 17)
    O = oracle.Oracle(mi.cell_k(dims, 4, -2, 2, seed=10), degree=10)
    x = mi.random_nodal(dims, 1)
    y = mi.random_nodal(dims, 2)
    Mx, My = O.vcycle(x), O.vcycle(y)
    assert abs(np.sum(Mx * y) - np.sum(x * My)) <= 1e-13 * np.sqrt(np.sum(Mx ** 2) * np.sum(y ** 2))


# ------------------------------------------------------------------ Galerkin
def prolongation_matrix(dims_f):
    """Trilinear P (fine interior x coarse interior) written from its
    definition: per axis a fine interior index 2c+1 is coarse node c (weight
    1), an index 2c lies halfway between coarse nodes c-1 and c (1/2 each)."""
    nf = [d - 2 for d in dims_f]           # (z, y, x) interior counts
    nc = [(n - 1) // 2 for n in nf]

    def axis(n_f, n_c):
        rows, cols, vals = [], [], []
        for g in range(n_f):
            if g % 2 == 1:
                rows.append(g); cols.append((g - 1) // 2); vals.append(1.0)
            else:
                for c in (g // 2 - 1, g // 2):
                    if 0 <= c < n_c:
                        rows.append(g); cols.append(c); vals.append(0.5)
        return sp.csr_matrix((vals, (rows, cols)), shape=(n_f, n_c))
    Pz, Py, Px = (axis(nf[a], nc[a]) for a in range(3))
    return sp.kron(sp.kron(Pz, Py), Px).tocsr()


def test_galerkin_operator_is_the_triple_product():
    """Coarse operators R A P with R = P^T/8, against scipy sparse products of
    an independently built P, on two successive levels (7-point fine operator,
    then a 27-point one)."""
    dims = (17, 17, 33)
    k = mi.cell_k(dims, 4, -2, 2, seed=41)
    O = oracle.Oracle(k, galerkin=True)
    A = dense_A(O, 0)
    d = dims
    for l in (1, 2):
        P = prolongation_matrix(d)
        ref = (P.T @ A @ P / 8.0).tocsr()
        got = dense_A(O, l)
        assert got.shape == ref.shape
        assert abs(got - ref).max() <= 1e-12 * abs(ref).max()
        assert got.nnz <= 27 * got.shape[0]
        A = got
        d = tuple((n - 1) // 2 + 1 for n in d)


def test_galerkin_coarse_correction_annihilates_the_restricted_residual():
    """With A_c = R A P an exact coarse-grid correction leaves a residual whose
    restriction vanishes: R (b - A (x + P A_c^-1 R (b - A x))) = 0.  (A
    re-discretised coarse operator does not have this property.)"""
    dims = (9, 17, 17)
    k = mi.cell_k(dims, 2, -2, 2, seed=42)
    b = mi.random_nodal(dims, 1)
    x = mi.random_nodal(dims, 2)
    for galerkin, small in ((True, True), (False, False)):
        O = oracle.Oracle(k, levels=2, galerkin=galerkin)
        bc = O.residual_restrict(b, x)
        x2 = O.prolong_add(O.coarse_solve(bc), x)
        after = np.max(np.abs(O.residual_restrict(b, x2))) / np.max(np.abs(bc))
        assert (after < 1e-12) == small, (galerkin, after)


def test_galerkin_chebyshev_interval_is_the_gershgorin_bound():
    dims = (33, 33, 33)
    k = mi.cell_k(dims, 4, -3, 3, seed=43)
    O = oracle.Oracle(k, galerkin=True)
    assert O.level_beta(0) == 2.0
    for l in range(1, O.levels):
        A = dense_A(O, l)
        g = np.max(np.asarray(abs(A).sum(axis=1)).ravel() / A.diagonal())
        assert abs(O.level_beta(l) - g) <= 1e-13 * g


def test_galerkin_pcg_matches_scipy_cg_and_beats_rediscretisation_at_high_contrast():
    dims = (33, 33, 33)
    k = mi.cell_k(dims, 4, -3, 3, seed=44)
    f = mi.rhs_f(dims, 44)
    O = oracle.Oracle(k, galerkin=True)
    x, it, info = O.pcg(f, 1e-10)
    A = dense_A(O)
    n = A.shape[0]

    def Minv(r):
        full = np.zeros(dims)
        full[1:-1, 1:-1, 1:-1] = r.reshape(31, 31, 31)
        return interior(O.vcycle(full)).ravel()

    count = [0]
    xs, flag = spla.cg(A, interior(f).ravel(), rtol=1e-10, atol=0.0, M=spla.LinearOperator((n, n), matvec=Minv),
                       maxiter=400, callback=lambda xk: count.__setitem__(0, count[0] + 1))
    assert flag == 0 and abs(count[0] - it) <= 1
    _, it_r, _ = oracle.Oracle(k).pcg(f, 1e-10, maxit=2000)
    assert it < it_r


# ------------------------------------------------------------------ FGMRES
def test_fgmres_residuals_match_an_independent_gmres():
    """For the (linear, float64) V-cycle M, flexible GMRES without restart is
    right-preconditioned GMRES: its j-th residual norm is min ||b - A M y||
    over y in the Krylov space K_j(A M, b).  Here that minimum comes from an
    Arnoldi process with modified Gram-Schmidt written with numpy, and a
    least-squares solve, independent of the oracle's classical Gram-Schmidt
    and Givens rotations."""
    dims = (17, 17, 17)
    k = mi.cell_k(dims, 4, -2, 2, seed=51)
    f = mi.rhs_f(dims, 51)
    O = oracle.Oracle(k)
    x, it, info = O.fgmres(f, 1e-10, restart=40, maxit=12)
    A = dense_A(O)
    n = A.shape[0]

    def M(v):
        full = np.zeros(dims)
        full[1:-1, 1:-1, 1:-1] = v.reshape(15, 15, 15)
        return interior(O.vcycle(full)).ravel()

    b = interior(f).ravel()
    beta = np.linalg.norm(b)
    Q = [b / beta]
    Hm = np.zeros((13, 12))
    for j in range(12):
        w = A @ M(Q[j])
        for i in range(j + 1):
            Hm[i, j] = w @ Q[i]
            w = w - Hm[i, j] * Q[i]
        Hm[j + 1, j] = np.linalg.norm(w)
        Q.append(w / Hm[j + 1, j])
        e = np.zeros(j + 2)
        e[0] = beta
        yv, *_ = np.linalg.lstsq(Hm[:j + 2, :j + 1], e, rcond=None)
        ref = np.linalg.norm(e - Hm[:j + 2, :j + 1] @ yv) / beta
        assert abs(info["hist"][j + 1] - ref) <= 1e-8 * ref + 1e-14, (j, info["hist"][j + 1], ref)


def test_fgmres_exact_preconditioner_and_agreement_with_cg():
    """One level: the preconditioner is the exact Cholesky solve, so one
    FGMRES iteration solves the system; on a multigrid hierarchy FGMRES (with
    and without restarts) and CG reach the same solution, with non-increasing
    residual estimates."""
    dims = (9, 9, 9)
    k = mi.cell_k(dims, 2, -1, 1, seed=52)
    f = mi.rhs_f(dims, 52)
    O1 = oracle.Oracle(k, levels=1)
    x1, it1, info1 = O1.fgmres(f, 1e-12)
    assert it1 == 1 and info1["true_rel_resid"] < 1e-13
    dims = (33, 33, 33)
    k = mi.cell_k(dims, 4, -1, 1, seed=53)
    f = mi.rhs_f(dims, 53)
    O = oracle.Oracle(k)
    xc, itc, _ = O.pcg(f, 1e-11)
    for m in (30, 4):
        x, it, info = O.fgmres(f, 1e-11, restart=m)
        assert info["true_rel_resid"] <= 1.01e-11
        assert np.all(np.diff(info["hist"]) <= 1e-15)
        assert np.linalg.norm(x - xc) <= 1e-9 * np.linalg.norm(xc)


# ------------------------------------------------------------------ inexact coarse solve
def test_coarse_gmres_is_exact_in_n_steps_and_meets_its_tolerance():
    """GMRES on the n coarsest unknowns reproduces the exact (Cholesky / numpy)
    solve when allowed n steps and a tiny tolerance; with the truncated
    tolerance 1e-4 of Sec. 5 its true residual is at most 1e-4 ||b|| (the
    rotated residual norm equals the true one in exact arithmetic)."""
    dims = (17, 9, 17)
    k = mi.cell_k(dims, 2, -2, 2, seed=71)
    Oe = oracle.Oracle(k)
    L = Oe.levels - 1
    dc = Oe.level_dims(L)
    b = mi.random_nodal(dc, 4)
    A = dense_A(Oe, L).toarray()
    n = A.shape[0]
    x_np = np.linalg.solve(A, interior(b).ravel())
    Ox = oracle.Oracle(k, coarse_gmres=True, coarse_rtol=1e-14, coarse_maxit=n)
    x = interior(Ox.coarse_solve(b)).ravel()
    assert np.linalg.norm(x - x_np) <= 1e-10 * np.linalg.norm(x_np)
    Ot = oracle.Oracle(k, coarse_gmres=True)
    xt = interior(Ot.coarse_solve(b)).ravel()
    rb = interior(b).ravel()
    assert np.linalg.norm(rb - A @ xt) <= 1e-4 * np.linalg.norm(rb) * (1 + 1e-9)
    assert np.linalg.norm(xt - x_np) > 1e-12 * np.linalg.norm(x_np)  # it is inexact


# ------------------------------------------------------------------ eigenvalue estimate
def test_lanczos_estimate_matches_numpy_and_bounds_the_spectrum():
    """eig_mode 1: the Lanczos estimate of the largest eigenvalue of D^-1 A
    equals the one built here with numpy (10 steps of Jacobi-preconditioned CG
    from the seeded start vector u(20160424, 3, i) - 1/2, the Lanczos
    tridiagonal from the CG coefficients, numpy's eigvalsh), lies below the
    true largest eigenvalue (a Ritz value) and close to it; the level's
    Chebyshev interval becomes [0.1 L, 1.1 L]."""
    dims = (17, 17, 33)
    k = mi.cell_k(dims, 4, -2, 2, seed=61)
    O = oracle.Oracle(k, eig_mode=1)
    for l in range(O.levels - 1):
        A = dense_A(O, l).toarray()
        n = A.shape[0]
        D = np.diag(A)
        r = mi.uniform(20160424, 3, np.arange(n, dtype=np.uint64)) - 0.5
        z = r / D
        p = z.copy()
        rz = r @ z
        al, be = [], []
        for _ in range(min(10, n)):
            q = A @ p
            a = rz / (p @ q)
            r = r - a * q
            z = r / D
            rzn = r @ z
            al.append(a)
            be.append(rzn / rz)
            p = z + be[-1] * p
            rz = rzn
        m = len(al)
        Tm = np.zeros((m, m))
        for j in range(m):
            Tm[j, j] = 1 / al[j] + (be[j - 1] / al[j - 1] if j else 0.0)
            if j + 1 < m:
                Tm[j, j + 1] = Tm[j + 1, j] = np.sqrt(be[j]) / al[j]
        ref = np.max(np.linalg.eigvalsh(Tm))
        got = O.level_lanczos(l)
        assert abs(got - ref) <= 1e-10 * ref, (l, got, ref)
        lmax = np.max(np.linalg.eigvalsh(A / np.sqrt(np.outer(D, D))))
        assert 0.8 * lmax <= got <= lmax * (1 + 1e-12)
        assert abs(O.level_beta(l) - 1.1 * got) <= 1e-14 * got
        assert abs(O.level_alpha(l) - 0.1 * got) <= 1e-14 * got


# ------------------------------------------------------------------ transfers
def test_prolongation_exact_on_trilinear_functions():
    dims = (17, 17, 17)
    O = oracle.Oracle(np.ones((16, 16, 16)), levels=2)
    g = lambda z, y, x: (1 + 2 * x) * (3 - y) * (0.5 + z) + 0.7 * x * y - 0.2 * z
    cz, cy, cx = grid(O.level_dims(1))
    ec = g(cz, cy, cx)
    ec[0] = ec[-1] = 0; ec[:, 0] = ec[:, -1] = 0; ec[:, :, 0] = ec[:, :, -1] = 0
    xf = O.prolong_add(ec, np.zeros(dims))
    fz, fy, fx = grid(dims)
    exact = g(fz, fy, fx)
    # fine nodes whose interpolation stencil uses interior coarse nodes only
    sl = slice(2, 15)
    assert np.max(np.abs(xf[sl, sl, sl] - exact[sl, sl, sl])) <= 1e-13


def test_restriction_is_transpose_of_prolongation_over_8():
    dims = (17, 9, 33)
    k = mi.cell_k(dims, 4, -1, 1, seed=2)
    O = oracle.Oracle(k, levels=2)
    u = mi.random_nodal(dims, 3)
    v = mi.random_nodal(O.level_dims(1), 4)
    Ru = O.residual_restrict(u, np.zeros(dims))
    Pv = O.prolong_add(v, np.zeros(dims))
    assert abs(np.sum(Ru * v) - np.sum(u * Pv) / 8.0) <= 1e-13 * np.sum(np.abs(u))
    one = np.zeros(dims)
    one[1:-1, 1:-1, 1:-1] = 1
    R1 = O.residual_restrict(one, np.zeros(dims))
    assert np.max(np.abs(interior(R1) - 1.0)) <= 1e-15


# ------------------------------------------------------------------ coarse solve
def test_coarsest_cholesky_matches_numpy():
    dims = (33,) * 3
    k = mi.cell_k(dims, 8, -1, 1, seed=1)
    O = oracle.Oracle(k)
    A, L = O.coarse_dense()
    Ac = dense_A(O, O.levels - 1).toarray()
    assert A.shape == (27, 27)
    np.testing.assert_array_equal(A, Ac)
    np.testing.assert_allclose(L @ L.T, A, rtol=0, atol=1e-14 * np.abs(A).max())
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=0, atol=1e-13 * np.abs(L).max())
    b = mi.random_nodal(O.level_dims(O.levels - 1), 9)
    x = O.coarse_solve(b)
    np.testing.assert_allclose(interior(x).ravel(), np.linalg.solve(A, interior(b).ravel()), rtol=1e-12)


# ------------------------------------------------------------------ V-cycle / PCG
def test_vcycle_symmetric_positive_definite():
    dims = (17, 17, 17)
    k = mi.cell_k(dims, 4, -2, 2, seed=8)
    O = oracle.Oracle(k)
    x = mi.random_nodal(dims, 1)
    y = mi.random_nodal(dims, 2)
    Mx, My = O.vcycle(x), O.vcycle(y)
    assert abs(np.sum(Mx * y) - np.sum(x * My)) <= 1e-13 * np.sqrt(np.sum(Mx ** 2) * np.sum(y ** 2))
    assert np.sum(Mx * x) > 0 and np.sum(My * y) > 0


def test_pcg_iterations_match_scipy_cg_with_same_preconditioner():
    dims = (17, 17, 17)
    k = mi.cell_k(dims, 4, -1, 1, seed=21)
    f = mi.rhs_f(dims, 21)
    O = oracle.Oracle(k)
    x, it, info = O.pcg(f, 1e-10)
    A = dense_A(O)
    n = A.shape[0]

    def Minv(r):
        full = np.zeros(dims)
        full[1:-1, 1:-1, 1:-1] = r.reshape(15, 15, 15)
        return interior(O.vcycle(full)).ravel()

    M = spla.LinearOperator((n, n), matvec=Minv)
    count = [0]
    xs, flag = spla.cg(A, interior(f).ravel(), rtol=1e-10, atol=0.0, M=M, maxiter=200,
                       callback=lambda xk: count.__setitem__(0, count[0] + 1))
    assert flag == 0
    assert abs(count[0] - it) <= 1
    assert np.max(np.abs(xs - interior(x).ravel())) <= 1e-8 * np.max(np.abs(xs))


def test_mesh_independent_iterations_constant_k():
    """Multigrid converges in a number of iterations independent of the mesh (Sec. 1)."""
    its = []
    for N in (9, 17, 33, 65):
        dims = (N,) * 3
        O = oracle.Oracle(np.ones((N - 1,) * 3))
        _, it, _ = O.pcg(mi.rhs_f(dims, 3), 1e-8)
        its.append(it)
    assert max(its) - min(its) <= 2, its


def test_flexible_and_standard_cg_agree_for_fp64_vcycle():
    dims = (17, 17, 17)
    k = mi.cell_k(dims, 4, -2, 2, seed=4)
    f = mi.rhs_f(dims, 4)
    O = oracle.Oracle(k)
    x1, it1, _ = O.pcg(f, 1e-10)
    x2, it2, _ = O.pcg(f, 1e-10, flexible=True)
    assert abs(it1 - it2) <= 1
    assert np.max(np.abs(x1 - x2)) <= 1e-8 * np.max(np.abs(x1))


def test_zero_rhs_and_nonconvergence():
    dims = (9, 9, 9)
    O = oracle.Oracle(np.ones((8, 8, 8)))
    x, it, info = O.pcg(np.zeros(dims), 1e-8)
    assert it == 0 and np.all(x == 0)
    x, it, info = O.pcg(mi.rhs_f(dims, 1), 1e-30, maxit=3)
    assert it == 3 and info["rel_resid"] > 0


# ------------------------------------------------------------------ gradient
def _loss_and_grad(O, f, phi_obs, mask, rtol=1e-13):
    phi, _, _ = O.pcg(f, rtol, maxit=400)
    g = np.where(mask, phi - phi_obs, 0.0)
    L = 0.5 * np.sum(g * (phi - phi_obs))
    lam, _, _ = O.pcg(g, rtol, maxit=400)
    return L, phi, lam


@pytest.mark.parametrize("face_rule", [0, 1])
def test_gradient_matches_central_differences(face_rule):
    dims = (9, 9, 9)
    lk = np.log(mi.cell_k(dims, 2, -1, 1, seed=31))
    f = mi.rhs_f(dims, 31)
    Oobs = oracle.Oracle(mi.cell_k(dims, 2, -1, 1, seed=32), face_rule=face_rule)
    phi_obs, _, _ = Oobs.pcg(f, 1e-13)
    mask = mi.obs_mask(dims, 31, frac=0.5)
    O = oracle.Oracle(np.exp(lk), face_rule=face_rule)
    L0, phi, lam = _loss_and_grad(O, f, phi_obs, mask)
    grad = O.gradient(phi, lam)
    rng = np.random.default_rng(0)
    cells = [tuple(rng.integers(0, 8, 3)) for _ in range(6)] + [(0, 0, 0), (7, 7, 7), (0, 3, 7)]
    h = 1e-6
    for c in cells:
        lp = lk.copy(); lp[c] += h
        lm = lk.copy(); lm[c] -= h
        Lp = _loss_and_grad(oracle.Oracle(np.exp(lp), face_rule=face_rule), f, phi_obs, mask)[0]
        Lm = _loss_and_grad(oracle.Oracle(np.exp(lm), face_rule=face_rule), f, phi_obs, mask)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(grad).max()), (c, fd, grad[c])


def test_adjoint_identities():
    dims = (17, 17, 17)
    k = mi.cell_k(dims, 4, -1, 1, seed=41)
    O = oracle.Oracle(k)
    f = mi.rhs_f(dims, 41)
    g = mi.random_nodal(dims, 42)
    Af, _, _ = O.pcg(f, 1e-13)
    Ag, _, _ = O.pcg(g, 1e-13)
    assert abs(np.sum(Af * g) - np.sum(f * Ag)) <= 1e-10 * np.sqrt(np.sum(Af ** 2) * np.sum(g ** 2))
    # dL/df = lambda for L = 0.5 |phi|^2; L is quadratic in f, so the central
    # difference (L(f+df) - L(f-df))/2 equals <lambda, df> up to solver error
    phi = Af
    lam, _, _ = O.pcg(phi, 1e-13)
    df = 1e-3 * mi.random_nodal(dims, 43)
    php, _, _ = O.pcg(f + df, 1e-13)
    phm, _, _ = O.pcg(f - df, 1e-13)
    dL = 0.25 * (np.sum(php ** 2) - np.sum(phm ** 2))
    assert abs(dL - np.sum(lam * df)) <= 1e-8 * abs(dL)


# ------------------------------------------------------------------ second summation order
# The oracle can run every dot product as a pairwise sum and every operator
# row in decreasing column order (sum_order=1).  The method fixes no
# summation order: sequential and pairwise float64 sums are both faithful
# readings of it.  The two fixed orders measure how far rounding order alone
# moves a solve, which is the evidence behind the GPU parity tolerances.
# These pins fix both orders against exact sums (math.fsum is correctly
# rounded) and their textbook error bounds.
def test_dot_products_in_both_orders_meet_their_error_bounds():
    u = 2.0 ** -53
    O0 = oracle.Oracle(np.ones((4, 4, 4)), levels=1)
    O1 = oracle.Oracle(np.ones((4, 4, 4)), levels=1, sum_order=1)
    rng = np.random.default_rng(11)
    differs = False
    for n in (1, 7, 8, 9, 1000, 100003):
        a = rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))
        b = rng.standard_normal(n)
        b[: n // 2] = -a[: n // 2] * (1.0 + 1e-3 * rng.standard_normal(n // 2))  # heavy cancellation
        exact = math.fsum(x * y for x, y in zip(a.tolist(), b.tolist()))  # products rounded once, as in both orders
        mag = float(np.sum(np.abs(a * b)))
        s0, s1 = O0.dot(a, b), O1.dot(a, b)
        assert abs(s0 - exact) <= n * u * mag * 1.01 + 1e-300
        assert abs(s1 - exact) <= (math.ceil(math.log2(max(n, 2))) + 8) * u * mag * 1.01 + 1e-300
        differs |= s0 != s1
    assert differs  # the second order is a different order, not the same sum again


def test_operator_rows_in_both_orders_meet_their_error_bounds():
    """Rows of A x summed in increasing and in decreasing column order: each
    within 7u sum_j |a_ij x_j| of the exact row sum of the same stored entries."""
    dims = (9, 17, 9)
    k = mi.cell_k(dims, 2, -3.0, 3.0, 12)
    O0 = oracle.Oracle(k, levels=1)
    O1 = oracle.Oracle(k, levels=1, sum_order=1)
    x = mi.random_nodal(dims, 13)
    rp, col, val = O0.csr()
    xi = interior(x).ravel()
    exact = np.array([math.fsum((val[q] * xi[col[q]]) for q in range(rp[p], rp[p + 1])) for p in range(len(rp) - 1)])
    mag = np.array([np.sum(np.abs(val[rp[p]:rp[p + 1]] * xi[col[rp[p]:rp[p + 1]]])) for p in range(len(rp) - 1)])
    y0 = interior(O0.apply(x)).ravel()
    y1 = interior(O1.apply(x)).ravel()
    u = 2.0 ** -53
    assert np.all(np.abs(y0 - exact) <= 7 * u * mag * 1.01)
    assert np.all(np.abs(y1 - exact) <= 7 * u * mag * 1.01)
    assert np.any(y0 != y1)


def test_second_summation_order_solves_the_same_problem():
    """Both orders run the same algorithm: on a moderate-contrast problem they
    take the same iterations to the same solution up to rounding."""
    dims = (17, 17, 17)
    k = mi.cell_k(dims, 4, -1.0, 1.0, 14)
    f = mi.rhs_f(dims, 14)
    x0, i0, _ = oracle.Oracle(k).pcg(f, 1e-10)
    x1, i1, _ = oracle.Oracle(k, sum_order=1).pcg(f, 1e-10)
    assert i0 == i1
    assert np.linalg.norm(x1 - x0) <= 1e-12 * np.linalg.norm(x0)
