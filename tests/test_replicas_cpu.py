"""The multi-GPU form is replicas only (independent slot batches, no
collective on the data path).  The benchmark's job summary -- max over ranks
of the step time, whole-job images / that time -- checked with 2 gloo ranks on
CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    value, ms = bench.replica_summary(mean_ms=2.0 + rank, images_per_rank=4096, dist=dist)
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_summary_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in got:
        assert ms == 3.0  # the slowest rank
        assert value == pytest.approx(2 * 4096 / 3e-3)


def test_replica_summary_single_process():
    import bench

    value, ms = bench.replica_summary(2.0, 4096)
    assert ms == 2.0 and value == pytest.approx(4096 / 2e-3)
