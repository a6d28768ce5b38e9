"""Predict-then-verify over a batch of instances: the learned path at scale.

    python -m paper_1609_05388_gb300.predict_verify --instances 4096 --predictor predictor.bin \
        [--compare 512] [--seed 7]

Instances come from the MNIST-shaped family (synth.mnist_like_family), n
log-uniform in [n_lo, n_hi], generated by a pool of worker processes started
with `spawn` before the first GPU call.  Batches of 64 go through
adagio_fit_batched with the dimension predictor: each instance's PCA gives its
spectrum features, the network guesses m, and one exhaustive certificate
verifies the guess; a failed guess falls back to the search from it.  The first
`--compare` instances are also fitted by the plain certified search, for the
dimension and time the guess saves or costs.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import time

import numpy as np

from . import synth


def _make(args):
    seed, n_lo, n_hi = args
    rng = np.random.default_rng(seed)
    n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
    return synth.mnist_like_family(rng, n)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=4096)
    ap.add_argument("--predictor", required=True)
    ap.add_argument("--compare", type=int, default=512)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--n-lo", type=int, default=2000)
    ap.add_argument("--n-hi", type=int, default=60000)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--workers", type=int, default=12)
    a = ap.parse_args()
    pool = mp.get_context("spawn").Pool(a.workers)
    jobs = [((a.seed + 1) * 2_000_003 + k, a.n_lo, a.n_hi) for k in range(a.instances)]
    stream = pool.imap(_make, jobs, chunksize=2)

    import torch
    from . import adagio as lib

    verified = fallback = not_cert = certs = 0
    m_learned, m_plain, gpu_s, gpu_plain_s = [], [], 0.0, 0.0
    with lib.Context(0) as ctx:
        ctx.mlp_load(a.predictor)
        done = 0
        while done < a.instances:
            items = [next(stream) for _ in range(min(a.batch, a.instances - done))]
            dX = [torch.from_numpy(X).cuda() for X, _ in items]
            epss = [e for _, e in items]
            torch.cuda.synchronize()
            t1 = time.time()
            res = ctx.fit_batched(dX, epss, graph=True, use_predictor=1)
            torch.cuda.synchronize()
            gpu_s += time.time() - t1
            for r in res:
                certs += r["full_certs"]
                if r["status"] != lib.OK:
                    not_cert += 1
                    m_learned.append(-1)
                    continue
                m_learned.append(r["m"])
                if r["probes"] == 1:
                    verified += 1
                else:
                    fallback += 1
            if done < a.compare:
                k = min(len(items), a.compare - done)
                torch.cuda.synchronize()
                t1 = time.time()
                res = ctx.fit_batched(dX[:k], epss[:k], graph=True)
                torch.cuda.synchronize()
                gpu_plain_s += time.time() - t1
                m_plain += [r["m"] if r["status"] == lib.OK else -1 for r in res]
            done += len(items)
            del dX
    pool.close()
    ml = np.array(m_learned[: len(m_plain)], dtype=np.float64)
    mp_ = np.array(m_plain, dtype=np.float64)
    both = (ml > 0) & (mp_ > 0)
    n_cmp = max(len(m_plain), 1)
    print(json.dumps({
        "instances": a.instances, "n_range": [a.n_lo, a.n_hi],
        "guess_verified_by_one_certificate": verified, "fallback_to_search": fallback,
        "not_certifiable": not_cert, "certificates": certs, "gpu_seconds": gpu_s,
        "instances_per_s": a.instances / gpu_s if gpu_s > 0 else None,
        "compared_with_plain_search": len(m_plain),
        "plain_search_gpu_seconds_on_those": gpu_plain_s,
        "learned_gpu_seconds_on_those_est": gpu_s * len(m_plain) / a.instances,
        "mean_ratio_learned_over_plain_m": float(np.mean(ml[both] / mp_[both])) if both.any() else None,
        "learned_below_plain": int(np.sum(ml[both] < mp_[both])),
        "learned_above_plain_by_more_than_10pct": int(np.sum(ml[both] > 1.1 * mp_[both])),
        "plain_per_instance_ms": 1e3 * gpu_plain_s / n_cmp}))


if __name__ == "__main__":
    main()
