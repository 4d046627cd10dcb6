"""Python binding of the multigrid-preconditioned CG library.

PyTorch supplies device memory and the current CUDA stream; every step of
the solve runs in the library's CUDA kernels (libmgpcg.so).  This module only
checks shapes, dtypes and devices and passes raw pointers through the C ABI.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import torch

from . import _lib as L


@dataclass
class Params:
    """Mirror of ``mg_params`` (include/mg.h); None keeps the library default."""
    levels: int = 0
    nu_pre: int = 1
    nu_post: int = 1
    cheby_degree: int = 2
    eig_lo_frac: float = 0.1
    eig_hi: float = 2.0
    coarse_k_rule: int = 0
    face_rule: int = 0
    precision: str = "fp64"
    maxit: int = 1000
    nonzero_guess: int = 0
    flexible: int = -1
    telescope_max_n: int = 4096
    use_graph: int = 1
    stencil_kernel: int = 0
    use_pdl: int = 1
    smoother: str = "chebyshev"  # or "richardson" (Jacobi-preconditioned, nu_pre / nu_post iterations)
    richardson_omega: float = 6.0 / 7.0
    coarse_op: str = "rediscretised"  # or "galerkin" (R A P, 27-point coarse stencils)
    krylov: str = "cg"  # or "fgmres" (flexible GMRES(gmres_restart), right-preconditioned)
    gmres_restart: int = 30
    eig_mode: int = 0  # 1: per-level Chebyshev interval from a 10-step Lanczos estimate
    eig_safety: float = 1.1
    coarse_solve: str = "cholesky"  # or "gmres" (Jacobi-preconditioned, to coarse_rtol; use krylov="fgmres")
    coarse_rtol: float = 1e-4
    coarse_maxit: int = 30
    bottom_blocks: int = 0  # 0 automatic; 1 one block; 2, 4, 8 a thread-block cluster
    test_inject: int = 0  # test only: 1 negated outer diagonal (breakdown), 2 negated coarsest diagonal (not SPD)
    slabs: int = 1  # z-slab decomposition of the solve (1: none)
    slab_level: int = 0  # agglomeration level of the slabs (0: the bottom kernel's first level)
    slab_rank: int = -1  # -1: this process holds all slabs; r: only slab r (one rank of a distributed solve)

    def to_c(self, k_is_log: bool) -> L.MgParams:
        p = L.MgParams()
        L.load().mg_params_default(C.byref(p))
        for name in ("levels", "nu_pre", "nu_post", "cheby_degree", "eig_lo_frac", "eig_hi", "coarse_k_rule",
                     "face_rule", "maxit", "nonzero_guess", "flexible", "telescope_max_n", "use_graph",
                     "stencil_kernel", "use_pdl", "richardson_omega"):
            setattr(p, name, getattr(self, name))
        p.smoother = {"chebyshev": 0, "richardson": 1}[self.smoother]
        p.coarse_op = {"rediscretised": 0, "galerkin": 1}[self.coarse_op]
        p.krylov = {"cg": 0, "fgmres": 1}[self.krylov]
        p.gmres_restart = self.gmres_restart
        p.eig_mode = self.eig_mode
        p.eig_safety = self.eig_safety
        p.coarse_solve = {"cholesky": 0, "gmres": 1}[self.coarse_solve]
        p.coarse_rtol = self.coarse_rtol
        p.coarse_maxit = self.coarse_maxit
        p.bottom_blocks = self.bottom_blocks
        p.test_inject = self.test_inject
        p.slabs = self.slabs
        p.slab_level = self.slab_level
        p.slab_rank = self.slab_rank
        p.precision = L.PRECISION[self.precision]
        p.k_is_log = 1 if k_is_log else 0
        return p


@dataclass
class Stats:
    iters: int
    rel_resid: float
    true_rel_resid: float
    bnorm: float
    setup_s: float
    solve_s: float
    kernel_launches: int = 0
    status: str = "MG_OK"
    history: list = field(default_factory=list)


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class MGSolver:
    """Level hierarchy for one conductivity field.

    ``k`` holds one value per finest cell, shape ``(Nz-1, Ny-1, Nx-1)``, as a
    float64 CUDA tensor (or ln k with ``k_is_log=True``).  Nodal tensors have
    shape ``(Nz, Ny, Nx)`` and live on the same device.
    """

    def __init__(self, k: torch.Tensor, params: Params | None = None, k_is_log: bool = False):
        self._lib = L.load()
        self._h = None
        if not (isinstance(k, torch.Tensor) and k.is_cuda and k.dtype == torch.float64 and k.dim() == 3):
            raise TypeError("k must be a 3-D float64 CUDA tensor")
        k = k.contiguous()
        self.device = k.device
        self.params = params or Params()
        self.cell_shape = tuple(k.shape)
        self.shape = tuple(s + 1 for s in k.shape)
        nz, ny, nx = self.shape
        h = C.c_void_p()
        cp = self.params.to_c(k_is_log)
        with torch.cuda.device(self.device):
            rc = self._lib.mg_setup(C.byref(h), nx, ny, nz, _ptr(k), 1, C.byref(cp), _stream())
        if rc != L.MG_OK:
            raise L.MgError(rc, self._lib.mg_last_error(None).decode())
        self._h = h

    def attach_transport(self, group=None):
        """For a handle built with slab_rank >= 0: connect it to the other
        ranks of the torch.distributed group (see slab_transport)."""
        from .slab_transport import SlabTransport
        self._transport = SlabTransport(self, group)
        return self._transport

    def close(self):
        if self._h is not None:
            self._lib.mg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- helpers
    def _check(self, rc: int):
        if rc != L.MG_OK:
            raise L.MgError(rc, self._lib.mg_last_error(self._h).decode())

    def _nodal(self, t: torch.Tensor, l: int = 0) -> torch.Tensor:
        shape = self.level_shape(l)
        if not (isinstance(t, torch.Tensor) and t.device == self.device and t.dtype == torch.float64
                and tuple(t.shape) == shape):
            raise ValueError(f"expected float64 tensor of shape {shape} on {self.device}")
        return t.contiguous()

    def _new(self, l: int = 0) -> torch.Tensor:
        return torch.empty(self.level_shape(l), dtype=torch.float64, device=self.device)

    def _sync_stream(self):
        self._check(self._lib.mg_set_stream(self._h, _stream())) if self._stream_changed() else None

    def _stream_changed(self) -> bool:
        s = _stream()
        if getattr(self, "_last_stream", None) != s:
            self._last_stream = s
            return True
        return False

    # -------------------------------------------------------------- info
    @property
    def num_levels(self) -> int:
        return self._lib.mg_num_levels(self._h)

    def level_shape(self, l: int):
        if l < 0:
            return self.shape
        N = (C.c_int * 3)()
        self._check(self._lib.mg_level_dims(self._h, l, N))
        return (N[2], N[1], N[0])

    def level_interval(self, l: int):
        """(alpha, beta): the Chebyshev interval of D^-1 A on level l."""
        a, b = C.c_double(), C.c_double()
        self._check(self._lib.mg_level_interval(self._h, l, C.byref(a), C.byref(b)))
        return a.value, b.value

    def history(self):
        n = self._lib.mg_history(self._h, None, 0)
        buf = (C.c_double * max(n, 1))()
        self._lib.mg_history(self._h, buf, n)
        return list(buf[:n])

    # -------------------------------------------------------------- solves
    def solve(self, f: torch.Tensor, rtol: float, x: torch.Tensor | None = None, raise_on_error: bool = True):
        """Return (x, Stats) for A x = f.  With raise_on_error=False the
        outcomes of the iteration itself (not converged, breakdown, a
        non-finite value, a device wait that gave up) come back in
        Stats.status instead of raising; argument, allocation and CUDA errors
        always raise."""
        f = self._nodal(f)
        x = self._new() if x is None else self._nodal(x)
        st = L.MgStats()
        self._sync_stream()
        rc = self._lib.mg_solve(self._h, _ptr(f), _ptr(x), float(rtol), C.byref(st))
        if rc != L.MG_OK and (raise_on_error or rc not in L.SOLVE_OUTCOMES):
            self._check(rc)
        return x, self._stats(st, rc)

    def solve_host(self, f: torch.Tensor, x: torch.Tensor, rtol: float, raise_on_error: bool = True) -> Stats:
        """Solve A x = f with f and x in HOST memory (float64 CPU tensors of the
        grid's shape; pinned memory gives full-bandwidth copies): the library
        copies f in and x out inside the call.  Returns the Stats; x is
        overwritten with the solution."""
        for t in (f, x):
            if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.dtype == torch.float64
                    and tuple(t.shape) == self.shape and t.is_contiguous()):
                raise ValueError(f"expected a contiguous float64 CPU tensor of shape {self.shape}")
        st = L.MgStats()
        self._sync_stream()
        rc = self._lib.mg_solve_host(self._h, _ptr(f), _ptr(x), float(rtol), C.byref(st))
        if rc != L.MG_OK and (raise_on_error or rc not in L.SOLVE_OUTCOMES):
            self._check(rc)
        return self._stats(st, rc)

    def solve_adjoint(self, g: torch.Tensor, rtol: float, phi: torch.Tensor | None = None, want_grad: bool = True):
        """Return (lambda, grad_logk or None, Stats) for A lambda = g."""
        g = self._nodal(g)
        lam = self._new()
        grad = torch.empty(self.cell_shape, dtype=torch.float64, device=self.device) if want_grad else None
        if want_grad:
            phi = self._nodal(phi)
        st = L.MgStats()
        self._sync_stream()
        rc = self._lib.mg_solve_adjoint(self._h, _ptr(g), _ptr(lam), float(rtol), _ptr(phi) if want_grad else None,
                                        _ptr(grad) if want_grad else None, C.byref(st))
        self._check(rc)
        return lam, grad, self._stats(st, rc)

    def _stats(self, st: L.MgStats, rc: int) -> Stats:
        return Stats(st.iters, st.rel_resid, st.true_rel_resid, st.bnorm, st.setup_s, st.solve_s,
                     st.kernel_launches, L.STATUS.get(rc, str(rc)), self.history())

    # -------------------------------------------------------------- steps
    def apply(self, x: torch.Tensor, level: int = 0) -> torch.Tensor:
        x = self._nodal(x, level)
        y = self._new(level)
        self._sync_stream()
        self._check(self._lib.mg_apply(self._h, level, _ptr(x), _ptr(y)))
        return y

    def smooth(self, b: torch.Tensor, x: torch.Tensor | None = None, level: int = 0) -> torch.Tensor:
        b = self._nodal(b, level)
        out = self._new(level) if x is None else self._nodal(x, level).clone()
        self._sync_stream()
        self._check(self._lib.mg_smooth(self._h, level, _ptr(b), _ptr(out), 1 if x is None else 0))
        return out

    def residual_restrict(self, b: torch.Tensor, x: torch.Tensor, level: int = 0) -> torch.Tensor:
        b, x = self._nodal(b, level), self._nodal(x, level)
        out = self._new(level + 1)
        self._sync_stream()
        self._check(self._lib.mg_residual_restrict(self._h, level, _ptr(b), _ptr(x), _ptr(out)))
        return out

    def prolong_add(self, ec: torch.Tensor, x: torch.Tensor, level: int = 0) -> torch.Tensor:
        ec = self._nodal(ec, level + 1)
        out = self._nodal(x, level).clone()
        self._sync_stream()
        self._check(self._lib.mg_prolong_add(self._h, level, _ptr(ec), _ptr(out)))
        return out

    def coarse_solve(self, b: torch.Tensor) -> torch.Tensor:
        l = self.num_levels - 1
        b = self._nodal(b, l)
        out = self._new(l)
        self._sync_stream()
        self._check(self._lib.mg_coarse_solve(self._h, _ptr(b), _ptr(out)))
        return out

    def vcycle(self, r: torch.Tensor) -> torch.Tensor:
        r = self._nodal(r)
        out = self._new()
        self._sync_stream()
        self._check(self._lib.mg_vcycle(self._h, _ptr(r), _ptr(out)))
        return out

    def gradient(self, phi: torch.Tensor, lam: torch.Tensor) -> torch.Tensor:
        phi, lam = self._nodal(phi), self._nodal(lam)
        out = torch.empty(self.cell_shape, dtype=torch.float64, device=self.device)
        self._sync_stream()
        self._check(self._lib.mg_gradient(self._h, _ptr(phi), _ptr(lam), _ptr(out)))
        return out

    def timing(self, on: bool = True, classes=None, levels=None):
        """Enable (and reset) or disable per-kernel device-time accounting,
        optionally only for the named kernel classes and the given levels."""
        cmask = 0
        if on:
            names = classes or L.KERNEL_CLASSES
            for n in names:
                cmask |= 1 << L.KERNEL_CLASSES.index(n)
        lmask = 0
        for l in (levels if levels is not None else range(31)):
            lmask |= 1 << l
        self._check(self._lib.mg_timing_enable(self._h, cmask, lmask))

    def kernel_times(self):
        """{(class, level): (ms, launches, points)} for classes with launches."""
        out = {}
        ms, n, pts = C.c_double(), C.c_longlong(), C.c_double()
        for ci, cname in enumerate(L.KERNEL_CLASSES):
            for l in range(self.num_levels):
                self._check(self._lib.mg_timing_read(self._h, ci, l, C.byref(ms), C.byref(n), C.byref(pts)))
                if n.value:
                    out[(cname, l)] = (ms.value, n.value, pts.value)
        return out

    def residual_norm(self, f: torch.Tensor, x: torch.Tensor) -> float:
        f, x = self._nodal(f), self._nodal(x)
        out = C.c_double()
        self._sync_stream()
        self._check(self._lib.mg_residual_norm(self._h, _ptr(f), _ptr(x), C.byref(out)))
        return out.value


class MGSolveFn(torch.autograd.Function):
    """phi = A(k)^-1 f with gradients with respect to f and per-cell ln k.

    forward(f, logk, params, rtol) builds the hierarchy from ln k and runs the
    forward solve; backward(dL/dphi) runs the adjoint solve A lambda = dL/dphi
    on the same (self-adjoint) operator and the fused face-flux gradient kernel,
    returning dL/df = lambda and dL/dln k.
    """

    @staticmethod
    def forward(ctx, f, logk, params: Params | None = None, rtol: float = 1e-10):
        solver = MGSolver(logk.detach(), params, k_is_log=True)
        phi, st = solver.solve(f.detach(), rtol)
        ctx.solver = solver
        ctx.rtol = rtol
        ctx.save_for_backward(phi)
        ctx.stats = st
        return phi

    @staticmethod
    def backward(ctx, gphi):
        (phi,) = ctx.saved_tensors
        # the solver stays open until ctx is collected (MGSolver.__del__ frees
        # it), so a second backward through the same graph works too
        lam, grad, _ = ctx.solver.solve_adjoint(gphi.contiguous(), ctx.rtol, phi, want_grad=ctx.needs_input_grad[1])
        return lam, grad, None, None


def mg_solve(f, logk, params: Params | None = None, rtol: float = 1e-10):
    """Differentiable solve: ``phi = mg_solve(f, logk)``."""
    return MGSolveFn.apply(f, logk, params, rtol)
