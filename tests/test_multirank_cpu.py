"""The benchmark's N > 1 path on CPU with the gloo backend (2 ranks).

Shots are independent, so the benchmark shards them (weak scaling) with no
collective on the data path; the one collective is the max over ranks of the
step time.  This test runs that host logic as two gloo processes.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from workloads import BB72, phenomenological_dem, sample_faults
    P = phenomenological_dem(BB72, 2, 0.01)
    per = 64
    first = bench.shard_first_shot(rank, per)
    F = sample_faults(P.p, 5, per, first_shot=first)
    ms = bench.reduce_max_ms(1.0 + rank, ws, torch.device("cpu"))
    rate = bench.aggregate_rate(ws, per, ms)
    q.put((rank, first, F, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_shots_and_reduce_the_step_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from workloads import BB72, phenomenological_dem, sample_faults
    P = phenomenological_dem(BB72, 2, 0.01)
    whole = sample_faults(P.p, 5, 128)
    (r0, f0, F0, ms0, rate0), (r1, f1, F1, ms1, rate1) = res
    assert (f0, f1) == (0, 64)
    assert np.array_equal(np.vstack([F0, F1]), whole)     # the shards tile the stream
    assert ms0 == ms1 == 2.0                              # both ranks see the slowest rank
    assert rate0 == rate1 == 2 * 64 / 2e-3
