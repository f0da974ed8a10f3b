"""The multi-rank reduction of bench.py (N > 1: independent replicas, value = all
fits / the slowest rank's time), run as two gloo ranks on the CPU."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank k took 10 + 5k ms and finished 20 - k fits
        ms, fits = bench.reduce_over_ranks(10.0 + 5.0 * rank, 20 - rank, "cpu")
        out[rank] = (ms, fits)
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (15.0, 39.0)  # max time, summed fits, on every rank


def test_reduce_over_ranks_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks(12.5, 7, "cpu") == (12.5, 7)
