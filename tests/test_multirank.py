"""The multi-rank path of bench.py (replicas: one independent problem per
rank, no data-path collective) on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # ranks report different step times and voxel counts
    ms_local = [2.0, 3.0][rank]
    vox_local = [1000, 3000][rank]
    ms_max, value = bench.aggregate_over_ranks(ms_local, vox_local)
    q.put((rank, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in res:
        assert ms_max == 3.0                              # max over ranks
        assert value == pytest.approx(4000 / 3e-3)        # all voxels / max time


def test_aggregate_single_rank():
    import bench
    ms, v = bench.aggregate_over_ranks(2.0, 1000)
    assert ms == 2.0 and v == pytest.approx(1000 / 2e-3)
