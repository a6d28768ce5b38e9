"""Trains the dimension predictor on instances labelled by the certified search.

    python -m paper_1609_05388_gb300.train_predictor --instances 2048 --out predictor.bin \
        [--record predictor.json] [--save-data labels.npz]

Instances come from the MNIST-shaped family (synth.mnist_like_family: rank,
cluster count, sparsity and eps vary) with n log-uniform in [n_lo, n_hi].
Batches of them are fitted with adagio_fit_batched: each is labelled with the
dimension the plain certified search returns (doubling and bisection with
exhaustive certificates) and its features come from the same fit's PCA.
Instances that are not certifiable at m = d carry no label and are dropped.
The network is trained full-batch with Adam on y = log m; the last
`--holdout` instances are kept out of training and reported.  Synthetic data
is generated by a pool of worker processes (started with `spawn`, before the
first GPU call) while the GPU labels the previous batch.  --record writes the
training record (instance counts, timings, holdout errors) as JSON beside the
weights; --save-data keeps the labelled features.
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
    ap.add_argument("--instances", type=int, default=2048)
    ap.add_argument("--holdout", type=int, default=128)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--n-lo", type=int, default=2000)
    ap.add_argument("--n-hi", type=int, default=60000)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=12)
    ap.add_argument("--out", required=True)
    ap.add_argument("--record", default="", help="write the training record (JSON) here")
    ap.add_argument("--save-data", default="", help="save the labelled features (npz) here")
    a = ap.parse_args()
    pool = mp.get_context("spawn").Pool(a.workers)
    jobs = [(a.seed * 1_000_003 + k, a.n_lo, a.n_hi) for k in range(a.instances)]
    stream = pool.imap(_make, jobs, chunksize=2)

    import torch
    from . import adagio as lib

    feats, labels, ns = [], [], []
    dropped = 0
    t0 = time.time()
    gpu_s = 0.0
    with lib.Context(0) as ctx:
        for b0 in range(0, a.instances, a.batch):
            items = [next(stream) for _ in range(min(a.batch, a.instances - b0))]
            t1 = time.time()
            dX = [torch.from_numpy(X).cuda() for X, _ in items]
            res = ctx.fit_batched(dX, [e for _, e in items], graph=True, features=True)
            torch.cuda.synchronize()
            gpu_s += time.time() - t1
            for (X, _), r in zip(items, res):
                if r["status"] != lib.OK:
                    dropped += 1
                    continue
                feats.append(r["feats"])
                labels.append(np.log(r["m"]))
                ns.append(X.shape[0])
            del dX
        label_s = time.time() - t0
        pool.close()
        F = np.array(feats, dtype=np.float32)
        t = np.array(labels, dtype=np.float32)
        if a.save_data:
            np.savez_compressed(a.save_data, feats=F, log_m=t, n=np.array(ns))
        N = len(t)
        tr = slice(0, N - a.holdout)
        ho = slice(N - a.holdout, N)
        ctx.mlp_init(a.seed)
        loss = float("nan")
        for it in range(a.steps):
            lr = 3e-3 if it < a.steps // 2 else (1e-3 if it < 3 * a.steps // 4 else 3e-4)
            loss = ctx.mlp_train_step(F[tr], t[tr], lr)
        y = ctx.mlp_forward(F[ho]).astype(np.float64)
        m_pred = np.ceil(1.05 * np.exp(y))
        m_true = np.exp(t[ho].astype(np.float64))
        ctx.mlp_save(a.out)
    rec = {"family": "synth.mnist_like_family", "n_range": [a.n_lo, a.n_hi], "seed": a.seed,
           "instances": a.instances, "labelled": N, "dropped_not_certifiable": dropped,
           "label": "dimension returned by the plain certified search (FP16x3 tiles)",
           "label_seconds": label_s, "gpu_label_seconds": gpu_s, "adam_steps": a.steps,
           "train_loss": loss, "holdout": a.holdout,
           "holdout_mean_abs_log_err": float(np.mean(np.abs(y - t[ho]))),
           "holdout_mean_ratio_pred_over_true": float(np.mean(m_pred / m_true)),
           "holdout_under_predicted": int(np.sum(m_pred < m_true)),
           "prediction_rule": "m = ceil(1.05 exp(y))"}
    if a.record:
        with open(a.record, "w") as f:
            json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
