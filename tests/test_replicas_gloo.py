"""Multi-rank host logic of bench.py (replicas: barrier, max-over-ranks time, whole-job
throughput) on CPU with the gloo backend and world_size 2.  No GPU."""

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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench

    w, r, local = bench.dist_env()
    reps = bench.Replicas(w, r, backend="gloo")
    reps.barrier()
    my_ms = 100.0 + 50.0 * r  # rank 1 is the slow one
    ms = reps.max_ms(my_ms)
    value = bench.aggregate_gbs(w, 1e9, 4, ms)
    reps.barrier()
    reps.close()
    out.put((r, w, local, ms, value))


def test_replicas_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, ms, value) in enumerate(res):
        assert rank == r and world == 2 and local == r
        assert ms == pytest.approx(150.0)  # max over ranks
        assert value == pytest.approx(2 * 1e9 * 4 / 0.150 / 1e9)  # both replicas' bytes / slowest time


def test_single_rank_needs_no_process_group():
    import bench

    reps = bench.Replicas(1, 0)
    reps.barrier()
    assert reps.max_ms(12.5) == 12.5
    assert bench.aggregate_gbs(1, 2e9, 3, 1000.0) == pytest.approx(6.0)
    reps.close()
