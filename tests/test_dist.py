"""Host logic of the multi-GPU bench path on CPU: world_size 2 over gloo.
Each rank takes its own index window, or its own element of the sequence
partitioned by an extra dimension (Sec. 2.5.1); no collective on the data
path, the only collective is the max over ranks of the step time."""
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


def _partition_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np

    import bench
    import oracle
    from paper_2307_15584_gb300 import inputs

    dist.init_process_group("gloo", rank=rank, world_size=world)
    q, p = bench.rank_partition(rank, world)
    W = oracle.sobol_matrices_wide(7, 64, inputs.sobol_raw_init(7))
    u, _ = oracle.sobol_points_partitioned(W, q, p, 0, 256, oracle.SCRAMBLE_NESTED, inputs.scramble_seeds(6),
                                           threads=1)
    parts = [None] * world
    dist.all_gather_object(parts, (p, u))  # test-only gather: the bench path has no data collective
    out[rank] = parts
    dist.destroy_process_group()


def test_partition_plan_rebuilds_the_sequence():
    """Two ranks, two elements: interleaved by their low index bit, the
    elements' rows are dimensions 1..6 of the whole sequence."""
    import numpy as np

    import oracle
    from paper_2307_15584_gb300 import inputs

    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_partition_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        parts = dict(out)[0]
    W = oracle.sobol_matrices_wide(7, 64, inputs.sobol_raw_init(7))
    seeds = np.concatenate([[0], inputs.scramble_seeds(6)]).astype(np.uint32)
    whole, _ = oracle.sobol_points_wide(W, 0, 512, oracle.SCRAMBLE_NESTED, seeds)
    rebuilt = np.empty((512, 6), np.uint32)
    for p, u in parts:
        rebuilt[p::2] = u  # q = 1: element p owns the indices 2J + p
    np.testing.assert_array_equal(rebuilt, whole[:, 1:])


def test_rank_partition_bounds():
    import bench

    assert bench.rank_partition(0, 1) == (0, 0)
    assert bench.rank_partition(5, 8) == (3, 5)
    for bad in ((0, 3), (2, 2), (0, 0)):
        with pytest.raises(ValueError):
            bench.rank_partition(*bad)
