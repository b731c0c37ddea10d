"""The N > 1 bench path on CPU: two gloo ranks, each timing its own replica; the job time is
the maximum over ranks and the value counts every rank's units (replicas only, no data-path
collective)."""
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
    local_ms = [100.0, 250.0][rank]  # rank 1 is the slow one
    value, max_ms = bench.aggregate(local_ms, units_per_rank=1000, dist=dist, device="cpu")
    dist.barrier()
    out[rank] = (value, max_ms)
    dist.destroy_process_group()


def test_two_rank_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, PORT, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    value, max_ms = res[0]
    assert max_ms == 250.0
    assert abs(value - 2 * 1000 / 0.25) < 1e-9


PORT = _free_port()
