"""CPU FP64 oracle for the multigrid-preconditioned CG solve (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package.  It wraps ``mg_oracle.c`` (plain C, binary64, no FMA
contraction, assembled CSR operators) through ctypes and shares no code with
the GPU library.  Every array argument is a full vertex grid ``[z][y][x]``
including the zero Dirichlet boundary.

The functions follow these passages of the paper: Eq. 1-2 (operator),
Algorithm 1 applied recursively (V-cycle), Sec. 2.1.1 (level components),
Sec. 4.3 (Chebyshev smoother preconditioned with Jacobi; Richardson-Jacobi,
Sec. 2.1.1 and Sec. 5), Sec. 1 and
Sec. 3.3.1 (exact coarse factorisation), Sec. 2.1 / 4.2 (CG with a relative
residual stopping test).  The gradient (adjoint) is not in the paper; it is
the standard discrete adjoint of the same operator.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB = os.path.join(_HERE, "libmgoracle.so")
_lib = None

_dptr = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        vp = C.c_void_p
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, _dptr, C.c_int, C.c_int, C.c_int,
                                   C.c_int, C.c_double, C.c_double, C.c_int, C.c_int]
        lib.orc_create_opt.restype = vp
        lib.orc_create_opt.argtypes = [C.c_int, C.c_int, C.c_int, _dptr, C.c_int, C.c_int, C.c_int,
                                       C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int]
        lib.orc_level_beta.restype = C.c_double
        lib.orc_level_beta.argtypes = [vp, C.c_int]
        lib.orc_level_alpha.restype = C.c_double
        lib.orc_level_alpha.argtypes = [vp, C.c_int]
        lib.orc_level_lanczos.restype = C.c_double
        lib.orc_level_lanczos.argtypes = [vp, C.c_int]
        lib.orc_set_coarse.restype = C.c_int
        lib.orc_set_coarse.argtypes = [vp, C.c_int, C.c_double, C.c_int]
        lib.orc_set_eig_mode.restype = C.c_int
        lib.orc_set_eig_mode.argtypes = [vp, C.c_int, C.c_double]
        lib.orc_free.argtypes = [vp]
        lib.orc_num_levels.argtypes = [vp]
        lib.orc_level_dims.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        lib.orc_nnz.restype = C.c_long
        lib.orc_nnz.argtypes = [vp, C.c_int]
        lib.orc_csr.argtypes = [vp, C.c_int, np.ctypeslib.ndpointer(np.int64), np.ctypeslib.ndpointer(np.int32), _dptr]
        lib.orc_cells.argtypes = [vp, C.c_int, _dptr]
        lib.orc_coarse_n.argtypes = [vp]
        lib.orc_coarse_dense.argtypes = [vp, _dptr, _dptr]
        lib.orc_apply.argtypes = [vp, C.c_int, _dptr, _dptr]
        lib.orc_smooth.argtypes = [vp, C.c_int, _dptr, _dptr, C.c_int]
        lib.orc_residual_restrict.argtypes = [vp, C.c_int, _dptr, _dptr, _dptr]
        lib.orc_prolong_add.argtypes = [vp, C.c_int, _dptr, _dptr]
        lib.orc_coarse_solve.argtypes = [vp, _dptr, _dptr]
        lib.orc_vcycle.argtypes = [vp, C.c_int, _dptr, _dptr]
        lib.orc_pcg.restype = C.c_int
        lib.orc_pcg.argtypes = [vp, _dptr, _dptr, C.c_double, C.c_int, C.c_int, C.c_int, vp, _dptr]
        lib.orc_gradient.argtypes = [vp, _dptr, _dptr, _dptr]
        lib.orc_fgmres.restype = C.c_int
        lib.orc_fgmres.argtypes = [vp, _dptr, _dptr, C.c_double, C.c_int, C.c_int, vp, _dptr]
        lib.orc_set_smoother.restype = C.c_int
        lib.orc_set_smoother.argtypes = [vp, C.c_int, C.c_double]
        lib.orc_set_sum_order.restype = C.c_int
        lib.orc_set_sum_order.argtypes = [vp, C.c_int]
        lib.orc_dot.restype = C.c_double
        lib.orc_dot.argtypes = [vp, C.c_long, _dptr, _dptr]
        _lib = lib
    return _lib


def default_levels(dims, coarsest: int = 5) -> int:
    """Levels until the smallest axis reaches ``coarsest`` vertices (3 interior)."""
    N = list(dims)
    L = 1
    while all((n - 1) % 2 == 0 and (n - 1) // 2 + 1 >= coarsest for n in N):
        N = [(n - 1) // 2 + 1 for n in N]
        L += 1
    return L


class Oracle:
    """Multigrid hierarchy on the CPU.  ``dims = (N_z, N_y, N_x)`` vertices."""

    def __init__(self, k_cells, levels: int | None = None, nu_pre: int = 1, nu_post: int = 1,
                 degree: int = 2, eig_lo_frac: float = 0.1, eig_hi: float = 2.0,
                 coarse_rule: int = 0, face_rule: int = 0, smoother: int = 0, omega: float = 6.0 / 7.0,
                 galerkin: bool = False, eig_mode: int = 0, eig_safety: float = 1.1, coarse_gmres: bool = False,
                 coarse_rtol: float = 1e-4, coarse_maxit: int = 30, sum_order: int = 0):
        """smoother 0: Chebyshev(degree)-Jacobi sweeps; 1: Richardson-Jacobi
        iterations x += omega D^-1 (b - A x), nu_pre / nu_post of them.
        galerkin: coarse operators R A P instead of re-discretisation.
        eig_mode 1: per-level Chebyshev interval [eig_lo_frac L, eig_safety L]
        from a 10-step Lanczos estimate L of the largest eigenvalue of D^-1 A.
        coarse_gmres: inexact coarsest solve, GMRES with Jacobi to coarse_rtol.
        sum_order 1: the second fixed summation order (pairwise dot products,
        operator rows summed in decreasing column order), for measuring how
        much rounding order alone moves a solve."""
        lib = _load()
        k = np.ascontiguousarray(k_cells, dtype=np.float64)
        self.dims = tuple(s + 1 for s in k.shape)
        self.levels = levels if levels is not None else default_levels(self.dims)
        nz, ny, nx = self.dims
        self._h = lib.orc_create_opt(nx, ny, nz, k, self.levels, nu_pre, nu_post, degree, eig_lo_frac,
                                      eig_hi, coarse_rule, face_rule, 1 if galerkin else 0)
        if not self._h:
            raise ValueError("oracle: invalid grid, levels or k field")
        self._lib = lib
        if lib.orc_set_smoother(self._h, smoother, omega) != 0:
            raise ValueError("oracle: invalid smoother")
        if eig_mode and lib.orc_set_eig_mode(self._h, eig_mode, eig_safety) != 0:
            raise ValueError("oracle: invalid eigenvalue-estimate mode")
        if coarse_gmres and lib.orc_set_coarse(self._h, 1, coarse_rtol, coarse_maxit) != 0:
            raise ValueError("oracle: invalid coarse-solve settings")
        if sum_order and lib.orc_set_sum_order(self._h, sum_order) != 0:
            raise ValueError("oracle: invalid summation order")

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.orc_free(self._h)
            self._h = None

    def level_beta(self, l: int) -> float:
        """Upper end of level l's Chebyshev interval."""
        return self._lib.orc_level_beta(self._h, l)

    def level_alpha(self, l: int) -> float:
        """Lower end of level l's Chebyshev interval."""
        return self._lib.orc_level_alpha(self._h, l)

    def level_lanczos(self, l: int) -> float:
        """Lanczos estimate of the largest eigenvalue of D^-1 A on level l."""
        return self._lib.orc_level_lanczos(self._h, l)

    def dot(self, a, b) -> float:
        """a . b (flattened) in this hierarchy's summation order."""
        a = np.ascontiguousarray(a, dtype=np.float64).ravel()
        b = np.ascontiguousarray(b, dtype=np.float64).ravel()
        return self._lib.orc_dot(self._h, a.size, a, b)

    def level_dims(self, l: int):
        N = (C.c_int * 3)()
        self._lib.orc_level_dims(self._h, l, N)
        return (N[2], N[1], N[0])

    def csr(self, l: int = 0):
        """(indptr, indices, data) of A_l over interior unknowns (x fastest)."""
        nz, ny, nx = (d - 2 for d in self.level_dims(l))
        n = nx * ny * nz
        nnz = self._lib.orc_nnz(self._h, l)
        rp = np.empty(n + 1, np.int64)
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz, np.float64)
        self._lib.orc_csr(self._h, l, rp, col, val)
        return rp, col, val

    def cells(self, l: int):
        d = self.level_dims(l)
        out = np.empty(tuple(s - 1 for s in d), np.float64)
        self._lib.orc_cells(self._h, l, out)
        return out

    def coarse_dense(self):
        n = self._lib.orc_coarse_n(self._h)
        A = np.empty((n, n)); Lf = np.empty((n, n))
        self._lib.orc_coarse_dense(self._h, A, Lf)
        return A, Lf

    def _z(self, l):
        return np.zeros(self.level_dims(l), np.float64)

    @staticmethod
    def _c(a):
        return np.ascontiguousarray(a, dtype=np.float64)

    def apply(self, x, l: int = 0):
        y = self._z(l)
        self._lib.orc_apply(self._h, l, self._c(x), y)
        return y

    def smooth(self, b, x=None, l: int = 0):
        """One smoother sweep; zero initial guess when x is None."""
        out = self._z(l) if x is None else self._c(x).copy()
        self._lib.orc_smooth(self._h, l, self._c(b), out, 1 if x is None else 0)
        return out

    def residual_restrict(self, b, x, l: int = 0):
        out = self._z(l + 1)
        self._lib.orc_residual_restrict(self._h, l, self._c(b), self._c(x), out)
        return out

    def prolong_add(self, ec, x, l: int = 0):
        out = self._c(x).copy()
        self._lib.orc_prolong_add(self._h, l, self._c(ec), out)
        return out

    def coarse_solve(self, b):
        out = self._z(self.levels - 1)
        self._lib.orc_coarse_solve(self._h, self._c(b), out)
        return out

    def vcycle(self, r, l: int = 0):
        out = self._z(l)
        self._lib.orc_vcycle(self._h, l, self._c(r), out)
        return out

    def pcg(self, f, rtol: float, maxit: int = 500, flexible: bool = False, x0=None):
        """Return (x, iterations, info) with info = rel/true residual, history."""
        x = self._z(0) if x0 is None else self._c(x0).copy()
        hist = np.zeros(maxit + 1)
        out = np.zeros(3)
        it = self._lib.orc_pcg(self._h, self._c(f), x, rtol, maxit, 1 if flexible else 0,
                               0 if x0 is None else 1, hist.ctypes.data, out)
        if it < 0:
            raise FloatingPointError("oracle CG breakdown (p.Ap <= 0)")
        return x, it, dict(rel_resid=out[0], true_rel_resid=out[1], bnorm=out[2], hist=hist[:it + 1])

    def fgmres(self, f, rtol: float, maxit: int = 500, restart: int = 30):
        """Flexible GMRES(restart) with the V-cycle as right preconditioner, from
        x = 0.  Return (x, iterations, info) as pcg does."""
        x = self._z(0)
        hist = np.zeros(maxit + 1)
        out = np.zeros(3)
        it = self._lib.orc_fgmres(self._h, self._c(f), x, rtol, maxit, restart, hist.ctypes.data, out)
        if it < 0:
            raise FloatingPointError("oracle FGMRES breakdown")
        return x, it, dict(rel_resid=out[0], true_rel_resid=out[1], bnorm=out[2], hist=hist[:it + 1])

    def gradient(self, phi, lam):
        """dL/d ln k per finest cell from the state phi and adjoint lambda."""
        out = np.empty(tuple(s - 1 for s in self.dims), np.float64)
        self._lib.orc_gradient(self._h, self._c(phi), self._c(lam), out)
        return out
