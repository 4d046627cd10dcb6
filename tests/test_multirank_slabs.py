"""The z-slab partition of the solve exercised by two CPU ranks (gloo).

The library's own plan (mg_slab_plan: host arithmetic, no device) gives each
rank its planes on every level above the agglomeration level.  Each rank holds
only its planes of a vector, swaps boundary planes with its neighbour as the
decomposed solve does (its last plane into the next slab's lower pad plane,
the next slab's first plane into its upper pad plane) and applies, on its
planes only, the operator (the oracle's CSR rows), the full-weighting
restriction and the trilinear prolongation; the agglomeration level is
gathered to rank 0 and scattered back with one halo plane per side; a dot
product is summed per rank and then across ranks.  Rank 0 reassembles every
result, which must equal the oracle's whole-grid result.  A halo plane that
was not exchanged, or a wrong plane range, changes the reassembled result.
"""
import ctypes as C
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

DIMS = (65, 33, 65)  # (Nz, Ny, Nx): 4 levels, agglomeration at level 2 (15 x 7 x 15 interior)
W = (0.25, 0.5, 0.25)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def slab_plan(dims, slabs, slab_level=0):
    """(agglomeration level, bounds[l][s]) from the library's plan."""
    from paper_1604_07163_gb300 import _lib
    lib = _lib.load()
    p = _lib.MgParams()
    lib.mg_params_default(C.byref(p))
    p.slabs, p.slab_level = slabs, slab_level
    buf = (C.c_int * 1024)()
    la = C.c_int()
    rc = lib.mg_slab_plan(dims[2], dims[1], dims[0], C.byref(p), buf, 1024, C.byref(la))
    if rc != 0:
        raise ValueError(lib.mg_last_error(None).decode())
    S = slabs
    return la.value, [list(buf[l * (S + 1):(l + 1) * (S + 1)]) for l in range(la.value + 1)]


def restrict_planes(rf, zc0, zc1, zf_lo):
    """Full weighting onto coarse interior planes [zc0, zc1) from fine full
    planes held as rf (full-plane index zf_lo first)."""
    Nzf, Nyf, Nxf = rf.shape[0], rf.shape[1], rf.shape[2]
    Nyc, Nxc = (Nyf - 1) // 2 + 1, (Nxf - 1) // 2 + 1
    out = np.zeros((zc1 - zc0, Nyc, Nxc))
    for kc in range(zc0, zc1):
        Kc = kc + 1
        acc = np.zeros((Nyc - 2, Nxc - 2))
        for c in (-1, 0, 1):
            for b in (-1, 0, 1):
                for a in (-1, 0, 1):
                    K = 2 * Kc + c - zf_lo
                    acc += W[c + 1] * W[b + 1] * W[a + 1] * rf[K, 2 + b:Nyf - 2 + b:2, 2 + a:Nxf - 2 + a:2][:Nyc - 2, :Nxc - 2]
        out[kc - zc0, 1:-1, 1:-1] = acc
    return out


def prolong_planes(ec, zf0, zf1, zc_lo, fine_shape):
    """Trilinear interpolation onto fine interior planes [zf0, zf1) from
    coarse full planes held as ec (full-plane index zc_lo first); coarse
    boundary values are zero."""
    _, Nyf, Nxf = fine_shape
    Nyc, Nxc = ec.shape[1], ec.shape[2]

    def axis_weights(Nf, Nc):
        M = np.zeros((Nf, Nc))
        for F in range(1, Nf - 1):
            for Cc in (F // 2, (F + 1) // 2):
                if 1 <= Cc <= Nc - 2:
                    M[F, Cc] = 1.0 if F == 2 * Cc else 0.5
        return M

    My, Mx = axis_weights(Nyf, Nyc), axis_weights(Nxf, Nxc)
    out = np.zeros((zf1 - zf0, Nyf, Nxf))
    for k in range(zf0, zf1):
        K = k + 1
        acc = np.zeros((Nyf, Nxf))
        for Kc in (K // 2, (K + 1) // 2):
            wz = 1.0 if K == 2 * Kc else 0.5
            if Kc < 1:
                continue
            acc += wz * (My @ ec[Kc - zc_lo] @ Mx.T)
        if K % 2 == 0:  # coincident plane counted once
            acc = My @ ec[K // 2 - zc_lo] @ Mx.T
        out[k - zf0] = acc
    return out


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    import scipy.sparse as sp
    import mg_inputs as mi
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        la, B = slab_plan(DIMS, world)
        k = mi.cell_k(DIMS, 4, -2.0, 2.0, 31)
        O = oracle.Oracle(k)
        res = {}

        def halo(local):
            """Swap boundary planes with the neighbours: local holds full
            planes z0 .. z1+1 of this rank's slab (index 0 and -1 are pads)."""
            reqs = []
            if rank + 1 < world:  # my last plane -> next's lower pad; next's first plane -> my upper pad
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(local[-2])), rank + 1))
                buf = torch.empty(local[-1].shape, dtype=torch.float64)
                reqs.append(dist.irecv(buf, rank + 1))
            if rank > 0:
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(local[1])), rank - 1))
                buf0 = torch.empty(local[0].shape, dtype=torch.float64)
                reqs.append(dist.irecv(buf0, rank - 1))
            for r in reqs:
                r.wait()
            if rank + 1 < world:
                local[-1] = buf.numpy()
            if rank > 0:
                local[0] = buf0.numpy()

        def gather_planes(mine, l):
            obj = [None] * world
            dist.all_gather_object(obj, mine)
            return obj

        for l in range(la):
            Nz, Ny, Nx = O.level_dims(l)
            nz, ny, nx = Nz - 2, Ny - 2, Nx - 2
            z0, z1 = B[l][rank], B[l][rank + 1]
            x = mi.random_nodal((Nz, Ny, Nx), 40 + l)  # every rank can make it; each keeps only its planes
            local = np.zeros((z1 - z0 + 2, Ny, Nx))
            local[1:-1] = x[z0 + 1:z1 + 1]
            halo(local)
            # operator rows of my planes, columns read from my planes and the two halo planes
            rp, col, val = O.csr(l)
            A = sp.csr_matrix((val, col, rp), shape=(nx * ny * nz, nx * ny * nz))
            rows = np.arange(z0 * nx * ny, z1 * nx * ny)
            xv = np.zeros(nx * ny * nz)
            lo, hi = max(z0 - 1, 0), min(z1 + 1, nz)
            xv[lo * nx * ny:hi * nx * ny] = local[lo - z0 + 1:hi - z0 + 1, 1:-1, 1:-1].ravel()
            y_mine = (A[rows] @ xv).reshape(z1 - z0, ny, nx)
            ys = gather_planes(y_mine, l)
            # restriction of my fine planes (with my upper halo) onto my coarse planes
            zc0, zc1 = B[l + 1][rank], B[l + 1][rank + 1]
            bc_mine = restrict_planes(local, zc0, zc1, z0)
            bcs = gather_planes(bc_mine, l)
            # prolongation onto my fine planes from my coarse planes (with my lower halo)
            Nzc, Nyc, Nxc = O.level_dims(l + 1)
            e = mi.random_nodal((Nzc, Nyc, Nxc), 60 + l)
            el = np.zeros((zc1 - zc0 + 2, Nyc, Nxc))
            el[1:-1] = e[zc0 + 1:zc1 + 1]
            halo(el)
            p_mine = prolong_planes(el, z0, z1, zc0, (Nz, Ny, Nx))
            ps = gather_planes(p_mine, l)
            # a dot product: per-rank sums, then across ranks in rank order
            part = float(np.sum(x[z0 + 1:z1 + 1] * x[z0 + 1:z1 + 1]))
            parts = [None] * world
            dist.all_gather_object(parts, part)
            if rank == 0:
                y = np.concatenate(ys)
                yo = O.apply(x, l)[1:-1, 1:-1, 1:-1]
                res[f"apply{l}"] = float(np.max(np.abs(y - yo)) / np.max(np.abs(yo)))
                bc = np.concatenate(bcs)
                bco = O.residual_restrict(x, np.zeros_like(x), l)[1:-1]
                res[f"restrict{l}"] = float(np.max(np.abs(bc - bco)) / np.max(np.abs(bco)))
                pf = np.concatenate(ps)
                po = O.prolong_add(e, np.zeros((Nz, Ny, Nx)), l)[1:-1]
                res[f"prolong{l}"] = float(np.max(np.abs(pf - po)) / np.max(np.abs(po)))
                res[f"dot{l}"] = abs(sum(parts) - float(np.sum(x * x))) / float(np.sum(x * x))
        # agglomeration: gather the level-la right-hand side to rank 0, scatter
        # the correction back with one halo plane on each side
        Nz, Ny, Nx = O.level_dims(la)
        z0, z1 = B[la][rank], B[la][rank + 1]
        b = mi.random_nodal((Nz, Ny, Nx), 70)
        g = [None] * world
        dist.all_gather_object(g, (z0, z1, b[z0 + 1:z1 + 1]))
        if rank == 0:
            full = np.zeros_like(b)
            for (a0, a1, planes) in g:
                full[a0 + 1:a1 + 1] = planes
            res["gather"] = float(np.max(np.abs(full - b)))
            xr = mi.random_nodal((Nz, Ny, Nx), 71)  # the root's correction
            for r in range(1, world):
                dist.send(torch.from_numpy(np.ascontiguousarray(xr[B[la][r]:B[la][r + 1] + 2])), r)
            mine = xr[z0:z1 + 2]
        else:
            buf = torch.empty((z1 - z0 + 2, Ny, Nx), dtype=torch.float64)
            dist.recv(buf, 0)
            mine = buf.numpy()
        xr_all = [None] * world
        dist.all_gather_object(xr_all, (z0, z1, mine))
        if rank == 0:
            res["scatter"] = max(float(np.max(np.abs(m - xr[a0:a1 + 2]))) for a0, a1, m in xr_all)
        out.put((rank, la, B, res))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_rank_results():
    from paper_1604_07163_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_plan_bounds_cover_every_level_and_nest(two_rank_results):
    (_, la, B, _), (_, la1, B1, _) = two_rank_results
    assert la == la1 == 2 and B == B1
    for l in range(la + 1):
        b = B[l]
        assert b[0] == 0 and all(b[s] < b[s + 1] for s in range(len(b) - 1))
        if l < la:  # fine planes are the coarse planes' children, the last slab also the final plane
            assert all(B[l][s] == 2 * B[l + 1][s] for s in range(len(b) - 1))
            assert B[l][-1] == 2 * B[l + 1][-1] + 1


def test_partitioned_operator_transfers_and_dots_equal_the_oracle(two_rank_results):
    res = two_rank_results[0][3]
    for l in range(2):
        assert res[f"apply{l}"] < 1e-14, res
        assert res[f"restrict{l}"] < 1e-14, res
        assert res[f"prolong{l}"] < 1e-14, res
        assert res[f"dot{l}"] < 1e-14, res
    assert res["gather"] == 0.0 and res["scatter"] == 0.0


def test_plan_rejects_impossible_partitions():
    from paper_1604_07163_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built")
    with pytest.raises(ValueError):
        slab_plan(DIMS, 16)  # 15 planes on the agglomeration level
    la, B = slab_plan(DIMS, 2, slab_level=1)
    assert la == 1 and B[1] == [0, 15, 31] and B[0] == [0, 30, 63]
