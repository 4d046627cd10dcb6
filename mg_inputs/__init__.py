"""Seeded synthetic inputs for the variable-coefficient Poisson solve.

This module holds only the input definition: a counter-based random
generator and the recipes that turn it into a cell conductivity field ``k``,
a nodal right-hand side ``f`` and an observation mask.  It contains none of
the solver's arithmetic, so both the CPU oracle tests and the GPU path draw
their inputs from here.

Generator (counter-based, stateless):

    splitmix64(x) = mix(x + 0x9E3779B97F4A7C15) with Vigna's SplitMix64
                    finaliser (shifts 30, 27, 31; multipliers
                    0xBF58476D1CE4E5B9, 0x94D049BB133111EB)
    u(seed, stream, idx) = (splitmix64(splitmix64(seed ^ (stream << 56)) ^ idx) >> 11) * 2^-53

which is a uniform double in [0, 1).

Recipes (the paper's workloads are PETSc's built-in problems; these synthetic
fields stand in for them with the shapes of the heat-conduction problem
-div(k grad phi) = f on the unit cube, Eq. 2):

* cells ``(N_z-1, N_y-1, N_x-1)``; cell ``(ck, cj, ci)`` lies in block
  ``(ck//B, cj//B, ci//B)`` with linear block index
  ``ib = (bk*nby + bj)*nbx + bi``; ``log10 k = a + (b-a)*u(seed, 0, ib)``;
* ``f`` at interior node with full-grid linear index
  ``p = (K*N_y + J)*N_x + I`` is ``-1 + 2*u(seed, 1, p)``; 0 on the boundary;
* the observation mask is ``u(seed, 2, p) < frac`` on interior nodes.

Arrays are C order ``[z][y][x]`` (x fastest), full vertex grids including the
Dirichlet boundary.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """SplitMix64 output for state ``x`` (numpy uint64 scalar or array)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, idx):
    """u(seed, stream, idx) in [0, 1) as float64 (idx: int or uint64 array)."""
    key = splitmix64(np.uint64(seed) ^ (np.uint64(stream) << np.uint64(56)))
    bits = splitmix64(key ^ np.asarray(idx, dtype=np.uint64))
    return (bits >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def cell_log10_k(dims, block: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """log10 k per cell for a vertex grid ``dims = (N_z, N_y, N_x)``."""
    nz, ny, nx = (d - 1 for d in dims)
    nbz, nby, nbx = (-(-n // block) for n in (nz, ny, nx))
    ib = np.arange(nbz * nby * nbx, dtype=np.uint64)
    lb = (lo + (hi - lo) * uniform(seed, 0, ib)).reshape(nbz, nby, nbx)
    lb = np.repeat(np.repeat(np.repeat(lb, block, 0), block, 1), block, 2)
    return np.ascontiguousarray(lb[:nz, :ny, :nx])


def cell_k(dims, block: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Conductivity per cell, k = 10**(log10 k)."""
    return np.power(10.0, cell_log10_k(dims, block, lo, hi, seed))


def _interior_field(dims, seed: int, stream: int, fn, dtype) -> np.ndarray:
    nz, ny, nx = dims
    out = np.zeros(dims, dtype=dtype)
    ii = np.arange(1, nx - 1, dtype=np.uint64)
    jj = np.arange(1, ny - 1, dtype=np.uint64)
    plane = (jj[:, None] * np.uint64(nx) + ii[None, :])
    for k in range(1, nz - 1):
        p = np.uint64(k * ny * nx) + plane
        out[k, 1:ny - 1, 1:nx - 1] = fn(uniform(seed, stream, p))
    return out


def rhs_f(dims, seed: int) -> np.ndarray:
    """f ~ U[-1, 1] at interior nodes, 0 on the boundary (float64)."""
    return _interior_field(dims, seed, 1, lambda u: -1.0 + 2.0 * u, np.float64)


def obs_mask(dims, seed: int, frac: float = 0.05) -> np.ndarray:
    """Boolean observation mask on interior nodes (u < frac)."""
    return _interior_field(dims, seed, 2, lambda u: u < frac, np.bool_)


def random_nodal(dims, seed: int, stream: int = 7) -> np.ndarray:
    """U[-1, 1] test vector on interior nodes, 0 on the boundary."""
    return _interior_field(dims, seed, stream, lambda u: -1.0 + 2.0 * u, np.float64)


# Workloads: vertex count per dimension, k block size, log10 k range, tolerance.
# Seeds are (workload index * 1000 + 1); the observation field uses seed + 1.
WORKLOADS = {
    "poisson33_fp64": dict(N=33, block=8, lo=-1.0, hi=1.0, rtol=1e-10, seed=1),
    "poisson257_c1e4": dict(N=257, block=16, lo=-2.0, hi=2.0, rtol=1e-8, seed=1001),
    "poisson513_c1e6": dict(N=513, block=16, lo=-3.0, hi=3.0, rtol=1e-8, seed=2001),
    "adjoint129": dict(N=129, block=8, lo=-1.0, hi=1.0, rtol=1e-10, seed=3001),
    "poisson1025_c1e6": dict(N=1025, block=32, lo=-3.0, hi=3.0, rtol=1e-8, seed=4001),
}


def workload(name: str, N: int | None = None):
    """Return (dims, k_cells, f, spec) for a named workload (optionally resized)."""
    spec = dict(WORKLOADS[name])
    if N is not None:
        spec["N"] = N
    dims = (spec["N"],) * 3
    k = cell_k(dims, spec["block"], spec["lo"], spec["hi"], spec["seed"])
    f = rhs_f(dims, spec["seed"])
    return dims, k, f, spec
