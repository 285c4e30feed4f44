"""Host logic of the multi-GPU bench path on CPU: world_size 2 over gloo.
Each rank takes its own index window (no collective on the data path); the
only collective is the max over ranks of the step time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    begin, count = bench.rank_window(r, w, 1 << 10)
    windows = [None] * w
    dist.all_gather_object(windows, (begin, count))
    t = torch.tensor([1.5 + r])  # this rank's elapsed time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out[rank] = (windows, float(t.item()))
    dist.destroy_process_group()


def test_rank_windows_and_max_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        windows, tmax = res[rank]
        assert tmax == 2.5
        assert windows == [(0, 1024), (1024, 1024)]  # disjoint, contiguous index windows


def test_rank_window_bounds():
    import bench

    b, c = bench.rank_window(3, 4)
    assert (b, c) == (3 << 24, 1 << 24)
    assert b + c <= 1 << 32  # every window stays inside the 32-bit index range up to 256 ranks
    with pytest.raises(TypeError):
        bench.rank_window()
