"""The z-slab solve run as separate processes, one per slab
(mg_params.slab_rank), exchanging halo planes, dot-product sums and the
agglomeration level only through the torch.distributed transport
(slab_transport; gloo here, staged through host memory).

The processes share the test's one GPU.  None of their kernels waits on
another process: every exchange is a host-side collective between kernel
launches, so the processes cannot deadlock on the device.  Each process
builds the whole-grid hierarchy, keeps its slab and writes only its planes of
x; the assembled solution must follow the single-process decomposed solve
(the same kernels; only the cross-rank sums are added in the transport's
order) and meet the oracle's bar.
"""
import ctypes as C
import datetime
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import mg_inputs as mi
import oracle
from oracle_orders import check_fp64_solve_against_both_oracle_orders

pytestmark = pytest.mark.gpu
DIMS, BLOCK, CONTRAST, SEED, RTOL = (65, 65, 65), 8, 1.5, 91, 1e-10


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def level0_bounds(dims, slabs, params):
    from paper_1604_07163_gb300 import _lib
    lib = _lib.load()
    p = params.to_c(False)
    p.slabs = slabs
    buf = (C.c_int * 1024)()
    la = C.c_int()
    assert lib.mg_slab_plan(dims[2], dims[1], dims[0], C.byref(p), buf, 1024, C.byref(la)) == 0
    return list(buf[:slabs + 1])


def _rank_main(rank, world, port, params_kw, out):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        import paper_1604_07163_gb300 as mg
        dev = torch.device("cuda:0")
        k = mi.cell_k(DIMS, BLOCK, -CONTRAST, CONTRAST, SEED)
        f = mi.rhs_f(DIMS, SEED)
        prm = mg.Params(maxit=500, slabs=world, slab_rank=rank, **params_kw)
        S = mg.MGSolver(torch.tensor(k, device=dev), prm)
        S.attach_transport()
        x, st = S.solve(torch.tensor(f, device=dev), RTOL)
        b = level0_bounds(DIMS, world, prm)
        z0, z1 = b[rank], b[rank + 1]
        out.put((rank, z0, z1, x[z0 + 1:z1 + 1].cpu().numpy(), st.iters, st.true_rel_resid, list(st.history)))
        S.close()
    except Exception as e:  # reported to the parent, which fails the test
        out.put((rank, "error", repr(e), None, None, None, None))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def run_ranks(world, params_kw):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, params_kw, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in res:
        assert r[1] != "error", r
    x = np.zeros(DIMS)
    for _, z0, z1, planes, _, _, _ in res:
        x[z0 + 1:z1 + 1] = planes
    return x, res


@pytest.mark.parametrize("world,params", [(2, {}), (3, {}), (3, dict(precision="mixed_fp32")),
                                          (2, dict(coarse_op="galerkin"))])
def test_multiprocess_slab_solve(gpu_lib, world, params):
    mg = gpu_lib
    x, res = run_ranks(world, params)
    its = {r[4] for r in res}
    assert len(its) == 1  # every rank ran the same iterations (the dots are summed over the ranks)
    itg = its.pop()
    assert len({r[5] for r in res}) == 1
    k = mi.cell_k(DIMS, BLOCK, -CONTRAST, CONTRAST, SEED)
    f = mi.rhs_f(DIMS, SEED)
    # the same decomposition in one process
    xs, sts = mg.MGSolver(torch.tensor(k, device="cuda:0"), mg.Params(maxit=500, slabs=world, **params)).solve(
        torch.tensor(f, device="cuda:0"), RTOL)
    assert sts.iters == itg
    # the transport adds the ranks' partial sums in its own order (gloo's
    # all-reduce), the single process in slab order: rounding-level drift
    assert np.linalg.norm(x - xs.cpu().numpy()) <= 1e-11 * np.linalg.norm(x)
    if params.get("precision", "fp64") == "fp64":
        check_fp64_solve_against_both_oracle_orders(x, itg, res[0][6], f, k, RTOL,
                                                    oracle_kw=dict(galerkin=params.get("coarse_op") == "galerkin"),
                                                    hist_its=10)
    else:
        true = np.linalg.norm((f - oracle.Oracle(k).apply(x))[1:-1, 1:-1, 1:-1]) / np.linalg.norm(f)
        assert true <= 1.01 * RTOL
