"""The multi-rank (N > 1) host path of bench.py on CPU: two gloo ranks on
127.0.0.1 exchange only the timing and unit scalars (slowest time, summed
units), as the GPU replicas do over NCCL."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, n = bench.reduce_ranks(1.0 + rank, 10.0 * (rank + 1), world, "cpu")
        out[rank] = (t, n)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_ranks_gloo_world2():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # every rank sees the slowest time (2 s) and all units (10 + 20)
    assert res == {0: (2.0, 30.0), 1: (2.0, 30.0)}


def test_reduce_ranks_single():
    import bench
    assert bench.reduce_ranks(1.5, 7.0, 1, "cpu") == (1.5, 7.0)
