"""Replica logic of the benchmark on CPU: two gloo ranks.

Multi-GPU runs are independent replicas (the path has no exchange step): each rank takes its
own signals and the step time is the slowest rank's.  This checks the signal ranges are
disjoint and cover the ranks' share, and that the max over ranks reaches every rank.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    B = 64
    start = bench.replica_start(rank, B)
    local = 10.0 + 3.0 * rank
    mx = bench.max_over_ranks(local, world, "cpu")
    out[rank] = (start, mx)
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    starts = sorted(out[r][0] for r in range(world))
    assert starts == [0, 64]                       # disjoint batches of 64 signals
    assert all(out[r][1] == 13.0 for r in range(world))   # the slowest rank's time on every rank
