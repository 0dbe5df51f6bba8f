"""Replicas on several ranks, run as two gloo processes on CPU: the benchmark's rank
logic (own seed per rank, job time = slowest rank, units summed over ranks) and the
independence of the replicas' inputs.  No GPU: the runs themselves stay on one GPU each
and never exchange data, so the only collective is the final timing reduction."""
import os
import socket

import pytest
import torch.distributed as dist
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
    assert (w, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, desc = bench.workload("scale", r)
        # a replica's timed region and the pairs it processed (rank 1 is slower)
        t_ms = 100.0 + 50.0 * r
        units = float(p["n_ions"] or 0) + 1000.0 * (r + 1)
        t_max, total = bench.job_totals(dist, t_ms, units, "cpu")
        out.put((r, p["seed"], desc, t_max, total, units))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_reduce_like_the_benchmark():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, d0, t0, tot0, u0), (r1, s1, d1, t1, tot1, u1) = res
    assert (r0, r1) == (0, 1)
    # independent replicas: own seeds, same workload
    assert s0 != s1 and d0 == d1
    # every rank sees the slowest rank's time and the whole job's units
    assert t0 == t1 == 150.0
    assert tot0 == tot1 == pytest.approx(u0 + u1)


def _failing_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from datetime import timedelta

    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=10))
    try:
        if rank == 1:
            raise RuntimeError("replica failed before its timing reduction")
        import bench

        try:
            bench.job_totals(dist, 1.0, 1.0, "cpu")
            out.put((rank, "completed"))
        except Exception as e:  # the peer is gone: the collective ends with an error
            out.put((rank, "error: " + type(e).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_a_failed_replica_ends_the_reduction_with_an_error():
    """a rank that dies between steps (on the host, no GPU involved) makes the other
    rank's timing collective fail within its timeout instead of hanging"""
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    r, status = out.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert r == 0 and status.startswith("error")
    assert procs[1].exitcode != 0
