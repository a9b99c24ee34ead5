"""bench.py's N > 1 reduction on two gloo ranks (CPU): the job's throughput is
the solves of all ranks over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, solved = bench.reduce_over_ranks(100.0 + 50.0 * rank, 64 * (rank + 1), world, device="cpu")
    out[rank] = (ms, solved)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_total_solves():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (150.0, 64 + 128)


def test_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks(12.5, 7, 1) == (12.5, 7)
