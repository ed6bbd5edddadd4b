"""The multi-rank path of bench.py on the CPU: two gloo ranks (replicas, no
exchange in the solve) agree on the slowest rank's time and report the
whole-job rate; a rank that fails before the collective ends the job with an
error on the others instead of a hang (a short process-group timeout)."""
import datetime
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ranks(rank, world, port, q, fail_rank):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    try:
        if rank == fail_rank:
            raise SystemExit(3)  # leaves before the collective, between steps
        local_ms = 100.0 + 50.0 * rank  # the ranks' own timed regions
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        q.put((rank, ms, bench.whole_job_rate(10, world, ms / 1e3)))
    except SystemExit:
        raise
    except Exception as e:  # the collective gave up on the missing rank
        q.put((rank, "error", type(e).__name__))
    finally:
        if rank != fail_rank:
            try:
                dist.destroy_process_group()
            except Exception:
                pass


def test_slowest_rank_and_whole_job_rate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_ranks, args=(r, world, port, q, -1)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=60) for _ in range(world))
    for p in procs:
        p.join(30)
    # every rank sees the slowest rank's 150 ms; 10 solves on each of 2 ranks
    assert [o[1] for o in out] == [150.0] * world
    assert all(abs(o[2] - world * 10 / 0.15) < 1e-9 for o in out)
    import bench

    assert bench.whole_job_rate(10, 1, bench.max_over_ranks(100.0) / 1e3) == pytest.approx(100.0)


def test_a_rank_that_leaves_ends_the_collective():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_ranks, args=(r, 2, port, q, 1)) for r in range(2)]
    for p in procs:
        p.start()
    rank, what, kind = q.get(timeout=90)
    for p in procs:
        p.join(60)
    assert rank == 0 and what == "error"
    assert procs[1].exitcode == 3

