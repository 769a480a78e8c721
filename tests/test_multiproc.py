"""The N > 1 path of bench.py on CPU: two gloo ranks reduce their step times
to the slowest rank's, the whole-job rate counts every rank's units, and
each rank draws its own synthetic slices (replicas, no data-path exchange)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, dist, device="cpu")
    rate = bench.whole_job_rate(8 * 3, world, ms_max)
    n, L, traj, slices = bench.make_slices(2, rank)
    out[rank] = (ms_max, rate, float(np.abs(slices[0]["x"]).sum()), float(np.abs(slices[0]["smaps"]).sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_slowest_and_draw_their_own_slices():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(rank_main, args=(world, free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 15.0
    assert abs(out[0][1] - 8 * 3 * 2 / 0.015) < 1e-6
    assert out[0][2] != out[1][2]               # rank-seeded phantoms differ
    assert out[0][3] != out[1][3]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.whole_job_rate(80, 1, 400.0) == 200.0
