"""The multi-GPU path on CPU: two gloo ranks shard the batched workload with no
data-path collective (weak scaling), and the timing reductions give the
job-level numbers bench.py reports."""
import os

import pytest


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2506_01099_gb300 import workloads as W

    ivs = bench.rank_intervals(rank, 64)
    mine = W.total_integers(ivs)
    total = bench.sum_over_ranks(world, float(mine))
    slowest = bench.max_over_ranks(world, float(rank + 1))
    out.put((rank, [(iv.lo, iv.hi, iv.kinds) for iv in ivs], mine, total, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_without_exchange():
    import multiprocessing as mp
    import socket

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, iv0, n0, t0, s0), (r1, iv1, n1, t1, s1) = res
    assert (r0, r1) == (0, 1)
    assert not set(iv0) & set(iv1)           # disjoint work, no shared interval
    assert t0 == t1 == float(n0 + n1)        # value counts every rank's integers
    assert s0 == s1 == 2.0                   # time = the slowest rank
    assert all(2**32 <= lo < 2**40 and 2**16 <= hi - lo <= 2**30 for lo, hi, _ in iv0 + iv1)


def _report_and_exit(out, result, code):
    # put() hands the result to a feeder thread: flush it before the process ends without
    # running the exit handlers (a process group whose peer is gone is not torn down)
    out.put(result)
    out.close()
    out.join_thread()
    os._exit(code)


def _lost_worker(rank, world, port, out):
    import time

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      BNX_BENCH_BACKEND="gloo", BNX_BENCH_PG_TIMEOUT_S="10")
    try:
        import bench

        ws, r, _ = bench.dist_init()
        bench.barrier(ws)  # both ranks up: the first step starts
    except Exception as e:  # noqa: BLE001 -- reported, so the test fails with the reason
        _report_and_exit(out, ("setup failed on rank %d: %r" % (rank, e), 0.0), 1)
    if r == 1:
        # the device is lost between steps: once the barrier has completed on both sides
        # (nothing of this rank is in flight), the process is gone
        time.sleep(1.0)
        os._exit(3)
    time.sleep(2.0)  # this rank's step
    t0 = time.time()
    try:
        bench.max_over_ranks(ws, 1.0)  # the job's timing reduction after the step
        result = ("no error", time.time() - t0)
    except Exception as e:  # noqa: BLE001 -- any error ends the wait, which is the point
        result = (type(e).__name__, time.time() - t0)
    _report_and_exit(out, result, 0)


def test_lost_rank_ends_the_next_reduction_with_an_error():
    """A rank whose device is lost leaves between steps (its process exits); the other
    rank learns of it on the host: its next timing reduction fails with an error within
    the process group's timeout instead of hanging (gloo ranks on CPU, no GPU)."""
    import multiprocessing as mp
    import socket

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_lost_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    what, waited = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert not what.startswith("setup failed"), what
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
    assert what != "no error", what
    assert waited < 60, waited
