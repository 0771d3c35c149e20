"""The benchmark's multi-rank timing (N > 1) on CPU: two gloo ranks.

With N GPUs the benchmark runs N independent replicas (one process per GPU)
and reports the slowest rank's time; the only cross-rank steps are a barrier
and a max-reduction of the step time.  This checks both with world size 2.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        bench._barrier(world)
        out[rank] = bench._max_over_ranks(world, 10.0 * (rank + 1))
        bench._barrier(world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        assert dict(out) == {0: 20.0, 1: 20.0}
