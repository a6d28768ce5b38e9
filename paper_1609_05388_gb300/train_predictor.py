"""Trains the dimension predictor on instances labelled by the certified search.

    python -m paper_1609_05388_gb300.train_predictor --instances 300 --out predictor.bin

Instances come from the MNIST-shaped family (synth.mnist_like_family: rank,
cluster count, sparsity and eps vary) with n log-uniform in [n_lo, n_hi]; each
is labelled with the dimension the plain certified search returns (gallop and
bisect with exhaustive certificates), its features come from adagio_features,
and the network is trained full-batch with Adam on y = log m.  The last
`--holdout` instances are kept out of training and reported.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import adagio as lib
from . import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=300)
    ap.add_argument("--holdout", type=int, default=30)
    ap.add_argument("--n-lo", type=int, default=2000)
    ap.add_argument("--n-hi", type=int, default=60000)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    rng = np.random.default_rng(a.seed)
    feats, labels, ns = [], [], []
    t0 = time.time()
    with lib.Context(0) as ctx:
        for k in range(a.instances):
            n = int(np.exp(rng.uniform(np.log(a.n_lo), np.log(a.n_hi))))
            X, eps = synth.mnist_like_family(rng, n)
            A, m, s, c, rc = ctx.fit(X, eps=eps, m_cap=X.shape[1], seed=1)
            feats.append(ctx.features(X, eps))
            labels.append(np.log(m))
            ns.append(n)
        label_s = time.time() - t0
        F = np.array(feats, dtype=np.float32)
        t = np.array(labels, dtype=np.float32)
        tr = slice(0, a.instances - a.holdout)
        ho = slice(a.instances - a.holdout, a.instances)
        ctx.mlp_init(a.seed)
        for it in range(a.steps):
            lr = 3e-3 if it < a.steps // 2 else (1e-3 if it < 3 * a.steps // 4 else 3e-4)
            loss = ctx.mlp_train_step(F[tr], t[tr], lr)
        y = ctx.mlp_forward(F[ho]).astype(np.float64)
        m_pred = np.ceil(1.05 * np.exp(y))
        m_true = np.exp(t[ho].astype(np.float64))
        ctx.mlp_save(a.out)
    print(json.dumps({"instances": a.instances, "label_seconds": label_s, "train_loss": loss,
                      "holdout_mean_abs_log_err": float(np.mean(np.abs(y - t[ho]))),
                      "holdout_mean_ratio_pred_over_true": float(np.mean(m_pred / m_true)),
                      "holdout_under_predicted": int(np.sum(m_pred < m_true))}))


if __name__ == "__main__":
    main()
