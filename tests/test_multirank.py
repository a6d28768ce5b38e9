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


def _oracle_part(X, Y, eps, rows, shard, nshards):
    """An oracle row-range certificate as a library part struct."""
    from oracle.certificate import certificate
    from paper_1609_05388_gb300 import adagio as lib
    o = certificate(X, Y, eps, rows=rows)
    p = lib.CertPartStruct()
    p.pairs, p.degenerate, p.violations, p.overflow = o.pairs, o.degenerate, o.violations, o.overflow
    p.recomputed = 0
    for b in range(lib.HIST_BINS):
        p.hist[b] = int(o.hist[b])
    p.sum, p.bound_sum = o.sum, 0.0
    p.max = o.max if o.pairs > o.degenerate else -1.0
    p.max_bound = 0.0
    p.argmax_i, p.argmax_j = (o.argmax_i, o.argmax_j) if o.pairs > o.degenerate else (-1, -1)
    p.hist_lo, p.hist_hi, p.eps = o.lo, o.hi, o.eps
    p.shard, p.nshards = shard, nshards
    return p


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import ctypes
    import numpy as np
    import torch.distributed as dist
    from paper_1609_05388_gb300 import adagio as lib
    from paper_1609_05388_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = synth.small(seed=0, n=500, d=16)
    Y = (wl.X @ np.random.default_rng(3).standard_normal((16, 6)).astype(np.float32) / np.sqrt(6))
    Y = Y.astype(np.float32)
    n = wl.X.shape[0]
    # this rank's part of the certificate, then every part on every rank
    part = _oracle_part(wl.X, Y, 0.2, (rank * n // world, (rank + 1) * n // world), rank, world)
    buf = torch.frombuffer(bytearray(bytes(part)), dtype=torch.uint8)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    structs = [lib.CertPartStruct.from_buffer_copy(bytes(t.numpy())) for t in parts]
    merged = lib.cert_merge(structs)
    q.put((rank, merged.pairs, merged.violations, merged.overflow, merged.degenerate,
           merged.hist.tolist(), merged.max, merged.argmax_i, merged.argmax_j, merged.mean))
    dist.destroy_process_group()


def test_certificate_parts_merge_over_two_gloo_ranks():
    """The certificate's combine step (adagio_cert_merge of per-rank parts,
    gathered over gloo) reproduces the whole certificate: counts, histogram,
    maximum and its pair exactly, the mean to rounding."""
    import numpy as np
    from oracle.certificate import certificate
    from paper_1609_05388_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = synth.small(seed=0, n=500, d=16)
    Y = (wl.X @ np.random.default_rng(3).standard_normal((16, 6)).astype(np.float32) / np.sqrt(6))
    o = certificate(wl.X, Y.astype(np.float32), 0.2)
    for (_, pairs, viol, over, deg, hist, mx, ai, aj, mean) in results:
        assert (pairs, viol, over, deg) == (o.pairs, o.violations, o.overflow, o.degenerate)
        assert hist == o.hist.tolist()
        assert (mx, ai, aj) == (o.max, o.argmax_i, o.argmax_j)
        assert abs(mean - o.sum / (o.pairs - o.degenerate)) <= 1e-12 * abs(mean)


def test_cert_merge_checks_its_parts():
    import numpy as np
    from paper_1609_05388_gb300 import adagio as lib
    from paper_1609_05388_gb300 import synth
    wl = synth.small(seed=1, n=300, d=8)
    Y = (1.1 * wl.X).astype(np.float32)
    parts = [_oracle_part(wl.X, Y, 0.2, (s * 100, (s + 1) * 100), s, 3) for s in range(3)]
    a = lib.cert_merge(parts)
    b = lib.cert_merge(parts[::-1])   # any order: merged in shard order
    assert (a.pairs, a.violations, a.max, a.argmax_i, a.mean) == \
        (b.pairs, b.violations, b.max, b.argmax_i, b.mean)
    assert (a.hist == b.hist).all()
    with pytest.raises(lib.AdagioError):
        lib.cert_merge(parts[:2])     # shard 2 of 3 missing
    dup = [parts[0], parts[0], parts[2]]
    with pytest.raises(lib.AdagioError):
        lib.cert_merge(dup)
    bad = _oracle_part(wl.X, Y, 0.3, (0, 100), 0, 3)
    with pytest.raises(lib.AdagioError):
        lib.cert_merge([bad, parts[1], parts[2]])  # another eps
