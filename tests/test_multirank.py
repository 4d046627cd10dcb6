"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

On several GPUs bench.py runs independent replicas: each rank solves its own
seeded problem and only the step time is combined (maximum over ranks).
These checks exercise that logic with two CPU processes.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import mg_inputs as mi
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = mi.WORKLOADS[bench.WORKLOAD]
    seed = bench.replica_seed(spec, rank)
    # each rank's problem is different; timing is the slowest rank's
    f = mi.rhs_f((9, 9, 9), seed)
    slowest = bench.max_over_ranks(10.0 + rank, torch.device("cpu"))
    value = bench.whole_job_dofs_per_s((spec["N"] - 2) ** 3, world, slowest)
    out.put((rank, seed, float(f.sum()), slowest, value, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, f0, t0, v0, e0), (r1, s1, f1, t1, v1, e1) = res
    assert s0 != s1 and f0 != f1          # independent problems
    assert t0 == t1 == 11.0               # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 255 ** 3 / 11.0e-3)
    assert e0 == (0, 2, 0) and e1 == (1, 2, 1)


def test_single_process_helpers_without_a_process_group():
    import torch
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_dofs_per_s(1000, 1, 1.0) == pytest.approx(1e6)
