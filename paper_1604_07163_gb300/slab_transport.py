"""Transport between the ranks of a z-slab solve over torch.distributed.

A handle built with mg_params.slab_rank = r holds only slab r of the
decomposed hierarchy; at its exchange points it calls three collective
operations (include/mg.h, mg_transport): the swap of halo planes with the
neighbouring ranks, the sum of the dot-product partial sums over the ranks,
and the all-gather of the agglomeration level.  This module implements them
with torch.distributed on device buffers it allocates:

- NCCL: the operations are issued on the library's own stream (as the
  current stream), so they are ordered with its kernels without the host
  waiting;
- gloo (CPU): the buffers are staged through host memory, the library's
  stream being synchronised before and the copies completed after.

It only moves bytes between the library's buffers; every step of the solve
runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import torch
import torch.distributed as dist

from . import _lib as L


class SlabTransport:
    def __init__(self, solver, group=None):
        lib = solver._lib
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.nccl = dist.get_backend(group) == "nccl"
        pb, bb = C.c_longlong(), C.c_longlong()
        rc = lib.mg_slab_transport_sizes(solver._h, C.byref(pb), C.byref(bb))
        if rc != L.MG_OK:
            raise L.MgError(rc, "the handle does not hold a single slab (slab_rank < 0)")
        self.plane_bytes, self.block_bytes = pb.value, bb.value
        dev = solver.device
        u8 = dict(dtype=torch.uint8, device=dev)
        self.send_lo = torch.zeros(self.plane_bytes, **u8)
        self.send_hi = torch.zeros(self.plane_bytes, **u8)
        self.recv_lo = torch.zeros(self.plane_bytes, **u8)
        self.recv_hi = torch.zeros(self.plane_bytes, **u8)
        self.red = torch.zeros(2, dtype=torch.float64, device=dev)
        self.gsend = torch.zeros(max(self.block_bytes, 1), **u8)
        self.grecv = torch.zeros(max(self.block_bytes, 1) * self.world, **u8)
        self.device = dev
        # the ctypes callbacks must outlive the handle's use of them
        self._cbs = (L.EXCHANGE_FN(self._exchange), L.ALLREDUCE_FN(self._allreduce),
                     L.ALLGATHER_FN(self._allgather))
        t = L.MgTransport(None, self._cbs[0], self._cbs[1], self._cbs[2], self.send_lo.data_ptr(),
                          self.send_hi.data_ptr(), self.recv_lo.data_ptr(), self.recv_hi.data_ptr(),
                          self.red.data_ptr(), self.gsend.data_ptr(), self.grecv.data_ptr())
        rc = lib.mg_set_transport(solver._h, C.byref(t))
        if rc != L.MG_OK:
            raise L.MgError(rc, lib.mg_last_error(solver._h).decode())

    def _stream(self, ptr):
        return torch.cuda.ExternalStream(ptr, device=self.device)

    # ---- halo planes with the neighbouring ranks
    def _exchange(self, ctx, nbytes, has_lo, has_hi, stream):
        try:
            n = int(nbytes)
            peers = []
            if has_lo:
                peers.append((self.send_lo[:n], self.recv_lo[:n], self.rank - 1))
            if has_hi:
                peers.append((self.send_hi[:n], self.recv_hi[:n], self.rank + 1))
            if self.nccl:
                with torch.cuda.stream(self._stream(stream)):
                    ops = []
                    for snd, rcv, peer in peers:
                        ops.append(dist.P2POp(dist.isend, snd, peer, self.group))
                        ops.append(dist.P2POp(dist.irecv, rcv, peer, self.group))
                    if ops:
                        for w in dist.batch_isend_irecv(ops):
                            w.wait()
            else:
                self._stream(stream).synchronize()
                reqs, outs = [], []
                for snd, rcv, peer in peers:
                    hs = snd.cpu()
                    hr = torch.empty_like(hs)
                    reqs.append(dist.isend(hs, peer, self.group))
                    reqs.append(dist.irecv(hr, peer, self.group))
                    outs.append((rcv, hr))
                for w in reqs:
                    w.wait()
                for rcv, hr in outs:
                    rcv.copy_(hr)
                torch.cuda.synchronize(self.device)
            return 0
        except Exception:  # a failure is reported to the library as a status, never raised through C
            return 1

    # ---- sum of the dot-product partials over the ranks
    def _allreduce(self, ctx, n, stream):
        try:
            v = self.red[:int(n)]
            if self.nccl:
                with torch.cuda.stream(self._stream(stream)):
                    dist.all_reduce(v, group=self.group)
            else:
                self._stream(stream).synchronize()
                h = v.cpu()
                dist.all_reduce(h, group=self.group)
                v.copy_(h)
                torch.cuda.synchronize(self.device)
            return 0
        except Exception:
            return 1

    # ---- the agglomeration level's blocks from every rank
    def _allgather(self, ctx, block_bytes, stream):
        try:
            b = int(block_bytes)
            if self.nccl:
                with torch.cuda.stream(self._stream(stream)):
                    dist.all_gather_into_tensor(self.grecv[:b * self.world], self.gsend[:b], group=self.group)
            else:
                self._stream(stream).synchronize()
                parts = [torch.empty(b, dtype=torch.uint8) for _ in range(self.world)]
                dist.all_gather(parts, self.gsend[:b].cpu(), group=self.group)
                self.grecv[:b * self.world].copy_(torch.cat(parts))
                torch.cuda.synchronize(self.device)
            return 0
        except Exception:
            return 1
