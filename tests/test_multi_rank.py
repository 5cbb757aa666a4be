"""The N > 1 path of the benchmark (replicas: one independent LP per rank, no
data-path collective; the job's time is its slowest rank's), run as two
`gloo` ranks on the CPU."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, _ = bench.dist_env()
        P = bench.make_problem("tiny", r)
        t_local = 10.0 + 5.0 * r                        # this rank's time, ms
        t_max = bench.max_over_ranks(t_local, w, device="cpu")
        value = bench.whole_job_rate(w, 100, t_max)
        solved_all = bench.sum_over_ranks(3 + 4 * r, w, device="cpu")   # LPs solved differ per rank
        dist.barrier()
        q.put((r, w, P.c[:4].tolist(), t_max, value, solved_all))
    finally:
        dist.destroy_process_group()


def test_replicas_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, c0, t0, v0, s0), (r1, w1, c1, t1, v1, s1) = out
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert not np.allclose(c0, c1)                      # each rank solves its own LP
    assert t0 == t1 == 15.0                             # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 100 / 0.015)   # all ranks' units over that time
    assert s0 == s1 == 10.0                             # the batch workload's solved LPs: 3 + 7


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1, 10, 1000.0) == pytest.approx(10.0)
    assert bench.sum_over_ranks(7, 1) == 7.0
