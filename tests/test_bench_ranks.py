"""The replica path of bench.py on CPU: two gloo ranks, each timing its own
copy of the job, reduce to the slowest rank's time and the summed units."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import importlib.util

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    seconds = [1.5, 2.25][rank]
    units = [100.0, 300.0][rank]
    out[rank] = bench.over_ranks(dist, seconds, units, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert dict(out) == {0: (2.25, 400.0), 1: (2.25, 400.0)}


@pytest.mark.parametrize("n", [1])
def test_over_ranks_single(n):
    """With one rank the figures pass through unchanged."""
    port = _free_port()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=0, world_size=n)
    try:
        import importlib.util

        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
        bench = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(bench)
        assert bench.over_ranks(dist, 3.0, 7.0, "cpu") == (3.0, 7.0)
    finally:
        dist.destroy_process_group()
