"""The residual-norm entry point that allocates nothing.

Some callers cannot allocate device memory when they check a solution, for
example because another memory manager owns the whole device, or because they
must keep a fixed footprint.  mg_residual_norm_noalloc serves them: its
scratch is a static device array held by the library.  This file checks,
through the C ABI, that it returns what mg_residual_norm returns, on two
calls in a row (the second call must not see stale partial sums).  It runs
last so that a failure here does not hide the other tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import mg_inputs as mi

pytestmark = pytest.mark.gpu


def test_noalloc_residual_norm_matches_existing_entry_point(gpu_lib):
    mg = gpu_lib
    from paper_1604_07163_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda:0")
    dims = (33, 17, 65)
    k = torch.tensor(mi.cell_k(dims, 4, -2.0, 2.0, 7), device=dev)
    S = mg.MGSolver(k)
    f = torch.tensor(mi.rhs_f(dims, 7), device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    f[:, 0] = -2.0  # boundary entries of f and x must be ignored by both entry points
    free_before = None
    for seed in (1, 2):  # two calls in a row with different x
        x = torch.tensor(mi.random_nodal(dims, seed), device=dev)
        x[0] = 5.0
        torch.cuda.synchronize()
        if seed == 2:  # after a first call: the second allocates nothing on the device
            free_before = torch.cuda.mem_get_info(dev)[0]
        rc = lib.mg_residual_norm_noalloc(S._h, f.data_ptr(), x.data_ptr(), out.data_ptr())
        assert rc == 0, lib.mg_last_error(S._h)
        torch.cuda.synchronize()
        if free_before is not None:
            assert torch.cuda.mem_get_info(dev)[0] == free_before
        got = out.item()
        ref = C.c_double()
        assert lib.mg_residual_norm(S._h, f.data_ptr(), x.data_ptr(), C.byref(ref)) == 0
        assert abs(got - ref.value) <= 1e-12 * ref.value, (seed, got, ref.value)
    # a converged solution gives a small residual through both paths
    f[:, 0] = 0.0
    xs, st = S.solve(f, 1e-10)
    lib.mg_residual_norm_noalloc(S._h, f.data_ptr(), xs.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    assert out.item() <= 1.01e-10 * np.linalg.norm(mi.rhs_f(dims, 7))
    S.close()


def test_noalloc_rejects_null_arguments(gpu_lib):
    from paper_1604_07163_gb300 import _lib
    lib = _lib.load()
    assert lib.mg_residual_norm_noalloc(None, None, None, None) == 1
