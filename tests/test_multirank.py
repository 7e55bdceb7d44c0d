"""The N>1 host logic on CPU: two gloo ranks, as bench.py runs replicas under torchrun.

Each rank replays its own trace (seed + rank, no data-path exchange); the job's
throughput is every rank's events over the slowest rank's time.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2212_07597_gb300 import tracegen as tg
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the replica's own work: its trace, seeded by rank, replayed alone
        tr = tg.plain_trace(20_000 + 5_000 * rank, seed=rank)
        o = oracle.Oracle(1_048_573, n_lines=256)
        o.replay_events(tr.delta, tr.addr, tr.line, tr.is_python)
        n_samples = len(o.samples())
        # made-up timings: rank r took 10 * (r + 1) ms for its events
        value, tmax = bench.job_throughput(10.0 * (rank + 1), tr.n)
        out[rank] = (value, tmax, tr.n, n_samples)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_events_over_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    total = res[0][2] + res[1][2]
    for r in range(world):
        value, tmax, _, _ = res[r]
        assert tmax == 20.0                      # the slowest rank's time
        assert np.isclose(value, total / 0.020)  # all ranks' events over it
    assert res[0][2] != res[1][2] and res[0][3] > 0 and res[1][3] > 0


def test_single_process_throughput_without_distributed():
    import bench
    v, t = bench.job_throughput(5.0, 1000)
    assert t == 5.0 and np.isclose(v, 200_000.0)
