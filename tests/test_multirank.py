"""The benchmark's multi-rank logic with two gloo ranks on the CPU.

With N GPUs the benchmark runs N independent replicas of the hot path (the
certificate of one data set is not split across GPUs): the ranks meet at
barriers around the timed region, the step time is the maximum over ranks and
the throughput the sum.  These are the only cross-rank steps; here they run on
two CPU processes over gloo, as torchrun would start them.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local, pg = bench.dist_setup(world)
    bench.barrier(pg)
    mx = bench.max_over_ranks(pg, 10.0 * (rank + 1))
    sm = bench.sum_over_ranks(pg, float(rank + 1))
    bench.barrier(pg)
    q.put((rank, r, w, local, mx, sm))
    pg.destroy_process_group()


def test_replica_reductions_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    for rank, (r_env, r, w, local, mx, sm) in enumerate(results):
        assert (r_env, r, w, local) == (rank, rank, 2, rank)
        assert mx == 20.0          # step time: the slowest rank
        assert sm == 3.0           # throughput: every rank's pairs


def test_single_process_needs_no_process_group():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    r, w, local, pg = bench.dist_setup(1)
    assert (r, w, pg) == (0, 1, None)
    assert bench.max_over_ranks(pg, 4.5) == 4.5 and bench.sum_over_ranks(pg, 4.5) == 4.5
