"""Multi-rank bench path on CPU: independent replicas, max-over-ranks time.

Lattices never exchange data (replicas only); the only collectives are the
barrier and the max of the per-rank timed region.  Run as two gloo ranks on
127.0.0.1 so the path is exercised without GPUs.
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), TLB_BENCH_BACKEND="gloo")
    import bench
    D, r, ws, local = bench.dist()
    assert (r, ws, local) == (rank, world, rank)
    D.barrier()
    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slow one
    ms = bench.max_over_ranks(D, ms_local, "cpu")
    value = bench.whole_job_mlups(1000 * 1000, 10, ws, ms)
    out.put((rank, ms, value))
    D.barrier()
    D.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, ms, value in res:
        assert ms == pytest.approx(150.0)
        # 2 ranks x 1e6 nodes x 10 steps in 150 ms
        assert value == pytest.approx(2 * 1e6 * 10 / 0.150 / 1e6)


def test_single_process_has_no_group():
    import bench
    assert bench.max_over_ranks(None, 12.5) == 12.5
    assert bench.whole_job_mlups(100, 10, 1, 1000.0) == pytest.approx(1e-3)
