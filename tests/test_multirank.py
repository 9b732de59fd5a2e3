"""The multi-rank (replicas) path of bench.py on CPU with the gloo backend, world size 2.

Each (frequency, source) system is independent, so every rank solves its own waves of frequencies
and ranks exchange only the timing: the slowest rank's time and the sums of the work counters.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    f = bench.rank_blocks(rank, world, 8, 4)
    ms = 100.0 + 50.0 * rank                 # rank 1 is the slow one
    out = bench.reduce_timing(ms, applies=10 * (rank + 1), solves=8, launches=70, world=world, dist=dist)
    q.put((rank, f, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_frequencies_and_reduce_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (f, o)) for r, f, o in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f0, o0 = res[0]
    f1, o1 = res[1]
    # replicas: each rank cycles through all four waves (the same mix of work), and at every step
    # the two ranks solve different waves
    assert sorted(f0) == sorted(f1) == [0, 0, 1, 1, 2, 2, 3, 3]
    assert all(a != b for a, b in zip(f0, f1))
    # both ranks see the same whole-job numbers: max time, summed work
    assert o0 == o1 == (150.0, 30.0, 16.0, 140.0)


def test_single_rank_passthrough():
    import bench
    assert bench.rank_frequencies(0, 1, 5, 32) == [0, 1, 2, 3, 4]
    assert bench.rank_frequencies(0, 1, 2, 32, per_wave=8) == list(range(16))
    assert bench.reduce_timing(12.5, 3, 2, 9, world=1) == (12.5, 3.0, 2.0, 9.0)


if __name__ == "__main__":  # pragma: no cover
    pytest.main([__file__])
