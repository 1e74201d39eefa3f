"""Host logic of bench.py's N > 1 path (one independent replica per rank):
max-over-ranks timing and the whole-job aggregate, on two gloo ranks (CPU)."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 180.0][rank]
    dist.barrier()
    ms = bench.max_over_ranks(local_ms, world, device="cpu")
    value = bench.aggregate_value(dof=1000, steps=4, seconds=ms * 1e-3, world=world)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_rank_timing_is_the_max_and_value_aggregates_all_replicas():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = out[r]
        assert ms == 180.0
        assert abs(value - 2 * 1000 * 4 / 0.180) < 1e-6


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_value(10, 2, 0.5, 1) == 40.0
