"""The N > 1 path of bench.py on CPU: gloo, world size 2, independent replicas.

Each rank solves its own (seeded) instance with the oracle on a tiny band and
the job time is the maximum over ranks (no data-path collective).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import time

    import numpy as np
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    from oracle.geometry import circle
    from oracle.multigrid import MGOptions, build_hierarchy, solve

    H = build_hierarchy(circle(), 1 / 32, 1 / 8, opts=MGOptions(smoother="jacobi"))
    b = H.fine.band
    _, f = synth.circle_fourier(b.cp[: b.nb], c=1.0 + rank)
    H2 = build_hierarchy(circle(), 1 / 32, 1 / 8, c=1.0 + rank, opts=MGOptions(smoother="jacobi"))
    t = time.perf_counter()
    u, rep = solve(H2, f, tol=1e-10)
    mine = time.perf_counter() - t + 0.05 * rank
    job = bench.max_over_ranks(mine, world)
    out[rank] = (rep.converged, mine, job)
    dist.destroy_process_group()


@pytest.mark.slow
def test_two_rank_replicas_max_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert all(res[r][0] for r in range(world))
    job = max(res[r][1] for r in range(world))
    assert all(abs(res[r][2] - job) < 1e-12 for r in range(world))
