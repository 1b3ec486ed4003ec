"""The multi-GPU path of the benchmark runs independent replicas (the cycle
does not shard; the ensemble of runs does): each rank times its own steps and
the job reports the slowest rank's time and the sum of all ranks' pushes.
Checked with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, n = bench.aggregate_replicas(100.0 + 50.0 * rank, 1000 * (rank + 1), world, "cpu")
    out[rank] = (t, n)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (150.0, 3000.0)


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_replicas(12.5, 7, 1, "cpu") == (12.5, 7)
