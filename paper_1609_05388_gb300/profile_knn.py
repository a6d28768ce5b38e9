"""Runs the k-nearest-neighbour graph of an embedded MNIST-shaped set, for profilers.

    python -m paper_1609_05388_gb300.profile_knn --n 60000 --m 421 --k 30

The points are Y = X A^T for a Gaussian A (m x 784); one adagio_knn call
builds the k-NN graph of the n points (Sec. 4.7's workload shape) after one
warm-up call on the first 1024 queries.  Prints one JSON line with the time
and the number of rows whose lists were re-searched exactly.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import adagio as lib
from . import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=60000)
    ap.add_argument("--m", type=int, default=421)
    ap.add_argument("--k", type=int, default=30)
    a = ap.parse_args()
    wl = synth.mnist_like(seed=1, n=a.n)
    A = (np.random.default_rng(0).standard_normal((a.m, wl.X.shape[1])) / np.sqrt(a.m)).astype(np.float32)
    with lib.Context(0) as ctx:
        Y = ctx.embed(A, torch.from_numpy(wl.X).cuda())
        ctx.knn(Y[:1024], a.k, B=Y)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.knn(Y, a.k)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        print(json.dumps({"n": a.n, "m": a.m, "k": a.k, "seconds": el,
                          "rows_searched_exactly": ctx.knn_last_exact_rows()}))


if __name__ == "__main__":
    main()
