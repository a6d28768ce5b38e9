"""Runs certified fits of the MNIST-shaped workload, for profilers.

    python -m paper_1609_05388_gb300.profile_fit --n 60000 --eps 0.1 --reps 1 [--learned] [--tol 1e-4]

Each repetition is one adagio_fit with the certified search (the benchmark's
step; with --learned, started from the shipped predictor's guess, as the
benchmark does).  Prints one JSON line with the fit statistics of the last
repetition.
"""
from __future__ import annotations

import argparse
import json
import os

import torch

from . import adagio as lib
from . import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=60000)
    ap.add_argument("--eps", type=float, default=0.1)
    ap.add_argument("--precision", default="fp16x3", choices=["fp32", "fp16x3", "bf16x3"])
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--learned", action="store_true")
    ap.add_argument("--tol", type=float, default=None, help="subspace-iteration tolerance")
    a = ap.parse_args()
    prec = {"fp32": lib.PREC_FP32, "fp16x3": lib.PREC_FP16X3, "bf16x3": lib.PREC_BF16X3}[a.precision]
    wl = synth.mnist_like(seed=1, n=a.n)
    X = torch.from_numpy(wl.X).cuda()
    with lib.Context(0) as ctx:
        if a.learned:
            ctx.mlp_load(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                      "predictor_mnist_like.bin"))
        for _ in range(a.reps):
            kw = {} if a.tol is None else {"tol": a.tol}
            A, m, s, c, rc = ctx.fit(X, eps=a.eps, m_cap=X.shape[1], seed=11, precision=prec,
                                     use_predictor=1 if a.learned else 0, **kw)
        st = ctx.last_fit_stats()
    print(json.dumps({"n": a.n, "eps": a.eps, "m": m, "s": s, "max": c.max, **st}))


if __name__ == "__main__":
    main()
