"""The multi-rank host logic of bench.py on two CPU ranks (gloo): each rank
shades its own frame of the orbit, the step time is the slowest rank's, and
the whole-job rate counts every rank's pixels."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        az, seed = bench.rank_frame(rank, world)
        frames = [None] * world
        dist.all_gather_object(frames, (az, seed))
        slowest = bench.max_over_ranks(1.5 + rank, torch.device("cpu"))
        dist.barrier()
        q.put((rank, frames, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_frames_and_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, frames, slowest in res:
        assert len(set(frames)) == world                  # every rank shades a different frame
        assert frames[0] == (0.0, 3)                       # rank 0: the single-GPU frame
        assert slowest == pytest.approx(1.5 + (world - 1))


def test_single_rank_and_whole_job_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_frame(0, 1) == (0.0, 3)
    assert bench.max_over_ranks(2.25, torch.device("cpu")) == 2.25
    # 4 ranks x 8,294,400 pixels in 2 ms -> 16.59 Gpixel/s
    assert bench.whole_job_rate(8294400, 4, 2.0) == pytest.approx(16.5888)
