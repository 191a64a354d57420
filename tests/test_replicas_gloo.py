"""The multi-GPU form is replicas only (independent maps, sessions and
keyframe windows; no exchange step): the benchmark's whole-job value is the
units all ranks processed over the slowest rank's time.  Checked here with
two gloo ranks on the CPU (the same host logic runs over NCCL on GPUs)."""
import multiprocessing
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, local = bench.dist_env()
        t, v = bench.replicas_value(1.0 + 0.5 * rank, 10.0, w, device="cpu")
        q.put((rank, r, w, local, t, v))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, r, w, local, t, v in res:
        assert (r, w, local) == (rank, 2, rank)
        assert t == 1.5                      # the slower rank's time
        assert v == pytest.approx(2 * 10.0 / 1.5)


def test_one_replica_needs_no_collective():
    import bench
    assert bench.replicas_value(2.0, 10.0, 1) == (2.0, 5.0)
