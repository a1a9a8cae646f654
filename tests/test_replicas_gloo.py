"""The multi-GPU form is replicas (one independent decomposition per rank, no
collective in the data path); the only cross-rank step is the bench's
aggregation: the slowest rank's time and the sum of all ranks' updates.
Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, upd = bench.aggregate_ranks(100.0 + 50.0 * rank, 1000.0 * (rank + 1), world, "cpu")
    q.put((rank, ms, upd))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, ms, upd in got:
        assert ms == 150.0 and upd == 3000.0


def test_aggregate_single_rank_is_identity():
    import bench
    assert bench.aggregate_ranks(12.5, 7.0, 1, "cpu") == (12.5, 7.0)
