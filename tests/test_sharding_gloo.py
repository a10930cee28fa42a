"""Multi-rank host logic of bench.py on CPU with two gloo ranks: every rank gets its own
batch of the same shape, the step time is the maximum over ranks, and the whole-job
throughput counts the tracks of all ranks (weak scaling, no data-path collective)."""

import os
import socket

import numpy as np
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


def _rank_main(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.make_workload("barrel", 1, rank, lo=200, hi=200)
        first = w.tracks.truth[0].tolist()
        firsts = [None] * world
        dist.all_gather_object(firsts, first)
        t_max = bench.max_over_ranks(0.010 * (rank + 1), dist, "cpu")
        thr = bench.aggregate_throughput(w.tracks.n_tracks, world, t_max)
        q.put((rank, firsts, t_max, thr, w.tracks.n_tracks))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    firsts = out[0][1]
    assert not np.allclose(firsts[0], firsts[1])        # distinct batches per rank
    for rank, _, t_max, thr, n in out:
        assert t_max == pytest.approx(0.020)              # the slowest rank's time
        assert thr == pytest.approx(world * n / 0.020)    # all ranks' tracks / slowest time
