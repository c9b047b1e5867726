"""The multi-GPU path of bench.py on CPU: two `gloo` ranks check that the
workload shards are disjoint and deterministic, that the step time is the
slowest rank's, that the whole-job value counts every rank's problems, and
that the reference arm runs on rank 0 only (replicas: no data-path
collective)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        seeds = [p.seed for p in bench.workload_problems(3, rank)]
        allseeds = [None] * world
        dist.all_gather_object(allseeds, seeds)
        t = bench.max_over_ranks(1.0 + rank, world)
        value = bench.whole_job_value(3, world, 4, t)

        class Args:
            gpus, steps, warmup = world, 1, 0
        ref = bench.run_reference(Args(), rank, world) if rank != 0 else None
        out.put((rank, allseeds, t, value, ref))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (_, seeds0, t0, v0, _), (_, seeds1, t1, v1, ref1) = res
    assert seeds0 == seeds1                                   # every rank sees the same shards
    a, b = seeds0
    assert len(a) == len(b) == 3 and not set(a) & set(b)      # disjoint
    import bench
    assert a == [p.seed for p in bench.workload_problems(3, 0)]   # deterministic
    assert t0 == t1 == 2.0                                    # the slowest rank's time
    assert v0 == v1 == 3 * 2 * 4 / 2.0                        # all ranks' problems
    assert ref1 is None                                       # reference arm: rank 0 only
