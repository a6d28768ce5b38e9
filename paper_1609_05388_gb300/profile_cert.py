"""Runs certificates of the MNIST-shaped workload at a chosen size, for profilers.

    python -m paper_1609_05388_gb300.profile_cert --n 16384 --m 400 --precision fp16x3 --reps 2 [--tiles pair]
    python -m paper_1609_05388_gb300.profile_cert --n 20000 --m 421 --prefixes 211,147,83,19

The embedding is Y = X A^T with A = [P ; S (I - P^T P)] at dimension m, built
from the library's PCA, JL matrix and assembly (no certificate runs before the
timed ones, so a profiler's first captured launches are theirs); each
repetition is one full adagio_distortion call (prep, tile kernel, recompute,
finaliser), or with --prefixes one adagio_distortion_prefixes call (the map's
certificate and the verdicts of the listed JL prefixes in one pass).  Prints
one JSON line with the per-stage times of the last repetition.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import adagio as lib
from . import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--m", type=int, default=400)
    ap.add_argument("--eps", type=float, default=0.1)
    ap.add_argument("--precision", default="fp16x3", choices=["fp32", "fp16x3", "bf16x3"])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--tiles", default="auto", choices=["auto", "single", "pair"],
                    help="tile kernel of the split-precision certificate")
    ap.add_argument("--band", type=int, default=0,
                    help="schedule band in tile rows (0: the default)")
    ap.add_argument("--prefixes", default="",
                    help="comma-separated JL prefix lengths for the multi-candidate certificate")
    a = ap.parse_args()
    prec = {"fp32": lib.PREC_FP32, "fp16x3": lib.PREC_FP16X3, "bf16x3": lib.PREC_BF16X3}[a.precision]
    wl = synth.mnist_like(seed=1, n=a.n)
    X = torch.from_numpy(wl.X).cuda()
    with lib.Context(0) as ctx:
        s = a.m // 2
        P, _ = ctx.pca(X, s, ctx.default_opts(seed=11))
        S = ctx.jl_matrix(11, a.m - s, X.shape[1])
        A = torch.from_numpy(ctx.assemble(P, S)).cuda()
        Y = ctx.embed(A, X)
        ctx.set_tile_kernel({"auto": lib.TILES_AUTO, "single": lib.TILES_SINGLE,
                             "pair": lib.TILES_PAIR}[a.tiles], a.band)
        ctx.set_timing(True)
        tile_ms = []
        kcs = [int(v) for v in a.prefixes.split(",") if v]
        verdicts = None
        for _ in range(a.reps):
            if kcs:
                c, res = ctx.distortion_prefixes(X, Y, s, a.eps, kcs, precision=prec)
                verdicts = [(r["k"], r["verdict"]) for r in res]
            else:
                c = ctx.distortion(X, Y, a.eps, precision=prec)
            tile_ms.append(ctx.last_cert_stats()["tile_ms"])
        st = ctx.last_cert_stats()
        kernel = ctx.tile_kernel_for(a.n)
    print(json.dumps({"n": a.n, "m": a.m, "precision": a.precision, "tiles": kernel,
                      "pairs": c.pairs, "max": c.max, "mean": c.mean,
                      "violations": c.violations, "recomputed": c.recomputed,
                      "tile_ms_all": tile_ms, "prefix_verdicts": verdicts, **st}))


if __name__ == "__main__":
    main()
