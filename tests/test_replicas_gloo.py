"""The multi-GPU path of the benchmark is replicas only: independent batches
per rank, no collective on the data path, and one max-reduction of the
ranks' timings.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank)
        q.put((rank, t, bench.replica_seed(100, rank)))
    finally:
        dist.destroy_process_group()


def test_replicas_take_max_time_and_distinct_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [t for _, t, _ in res] == [2.5, 2.5]
    assert res[0][2] != res[1][2]


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
