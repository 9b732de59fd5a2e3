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


def _solve_worker(rank, world, port, q):
    """Each rank solves the systems of its own waves (the bench's schedule) on a tiny grid with the
    oracle, then the ranks reduce the timing and the work counters as the bench does."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import time
    import numpy as np
    import bench
    import synthetic as sy
    from oracle import operator as op, solver as osv, source as osrc
    med = sy.random_medium((4, 5, 4), h=10.0, seed=80, frac=0.1)
    freqs = [3.0, 6.0, 9.0, 12.0, 15.0, 18.0, 21.0, 24.0]
    blocks = bench.freq_blocks(len(freqs), 2)
    seq = bench.rank_blocks(rank, world, 4, len(blocks))
    t0 = time.perf_counter()
    solved, iters = [], 0
    for blk in seq:
        for f in blocks[blk]:
            w = 2 * np.pi * freqs[f]
            u0, _ = osrc.background_field(med.n, med.h, sy.explosion(), np.array([14.0, 21.0, 13.0]), w,
                                          med.lam0, med.mu0, med.rho0)
            F = op.FFTOperator(med, w)
            x, it, rr, st, _ = osv.bicgstab(F.apply, u0, tol=1e-10, maxit=200)
            assert st == osv.OK and rr <= 1e-10
            solved.append(f)
            iters += it
    ms = 1e3 * (time.perf_counter() - t0)
    out = bench.reduce_timing(ms, applies=2 * iters, solves=len(solved), launches=0, world=world, dist=dist)
    q.put((rank, seq, solved, ms, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_solve_their_own_waves():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solve_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {r: rest for r, *rest in (q.get(timeout=300) for _ in procs)}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (seq0, sol0, ms0, out0), (seq1, sol1, ms1, out1) = res[0], res[1]
    # every rank solved all 8 frequencies once over its 4 waves, in a different order
    assert sorted(sol0) == sorted(sol1) == list(range(8))
    assert seq0 == [0, 1, 2, 3] and seq1 == [1, 2, 3, 0]
    # the whole-job numbers: the slower rank's time, the solves of both
    assert out0 == out1
    assert out0[0] == max(ms0, ms1) and out0[2] == 16.0


def test_single_rank_passthrough():
    import bench
    assert bench.rank_frequencies(0, 1, 5, 32) == [0, 1, 2, 3, 4]
    assert bench.rank_frequencies(0, 1, 2, 32, per_wave=8) == list(range(16))
    assert bench.reduce_timing(12.5, 3, 2, 9, world=1) == (12.5, 3.0, 2.0, 9.0)


if __name__ == "__main__":  # pragma: no cover
    pytest.main([__file__])
