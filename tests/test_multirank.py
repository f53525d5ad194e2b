"""The benchmark's multi-rank path on CPU: two ``gloo`` ranks.

Domains are independent replicas (no data-path collective); the only
cross-rank operations are the barriers around the timed region and the
max-over-ranks of the elapsed time, from which rank 0 forms the whole-job
throughput (cells of all ranks x steps / slowest rank's time).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        bench.barrier(ws)
        ms_local = 10.0 + 5.0 * rank  # the second rank is the slower one
        ms = bench.max_over_ranks(ms_local, ws)
        bench.barrier(ws)
        value = bench.whole_job_mlups(cells_per_rank=1000, ws=ws, steps=4, ms=ms)
        q.put((rank, env, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, ms, value in res:
        assert env == (ws, rank, rank)
        assert ms == pytest.approx(15.0)
        # 2 ranks x 1000 cells x 4 steps in 15 ms
        assert value == pytest.approx(2 * 1000 * 4 / 15e-3 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_mlups(cells_per_rank=10 ** 6, ws=1, steps=10, ms=2.0) == pytest.approx(5000.0)
