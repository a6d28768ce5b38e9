"""Dimension vs distortion of ADAGIO and its two baselines (Table 3, Fig. 6),
and of ADAGIO at several PCA accuracies (Sec. 4.5, Fig. 7).

    python -m paper_1609_05388_gb300.tradeoff --n 60000 [--eps 0.1 0.2 0.3] [--dims 25 50 100 200 400]
    python -m paper_1609_05388_gb300.tradeoff --n 60000 --pca-sweep 1e-6 1e-4 1e-3 1e-2

The three maps are ADAGIO (Sec. 4.1 split: floor(m/2) principal rows and the
rest JL rows), PCA only and JL only.  For each target distortion the certified
search returns the smallest dimension it finds (Table 3's "dimensions needed");
for each fixed dimension the exhaustive certificate gives the maximum and mean
distortion (Fig. 6's curves).  Every number comes from the tensor-core
certificate of the returned map.  Prints one JSON line per measurement.

--pca-sweep stands in for Fig. 7's exact vs randomized PCA: ADAGIO at each
fixed dimension with the subspace iteration stopped at each tolerance
(1e-6 is converged to FP32 accuracy and takes the place of the exact PCA;
looser tolerances stop after fewer iterations), with the certificate's max
and mean distortion and the PCA's time and iteration count.
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import adagio as lib
from . import synth

MODES = {"adagio": -1, "pca": None, "jl": 0}   # opts.s per mode (None: s = m_cap)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=60000)
    ap.add_argument("--eps", type=float, nargs="*", default=[0.1, 0.2, 0.3])
    ap.add_argument("--dims", type=int, nargs="*", default=[25, 50, 100, 200, 400])
    ap.add_argument("--tol", type=float, default=1e-3, help="subspace-iteration tolerance")
    ap.add_argument("--pca-sweep", type=float, nargs="*", default=None,
                    help="PCA tolerances of the Fig. 7 sweep (ADAGIO only, at --dims)")
    a = ap.parse_args()
    wl = synth.mnist_like(seed=1, n=a.n)
    X = torch.from_numpy(wl.X).cuda()
    d = X.shape[1]
    with lib.Context(0) as ctx:
        if a.pca_sweep:
            for m in a.dims:
                for tol in a.pca_sweep:
                    for _ in range(2):   # the second fit is the one timed
                        A, mm, s_out, c, rc = ctx.fit(X, eps=0.0, m=m, s=m // 2, seed=11,
                                                      precision=lib.PREC_FP16X3, tol=tol)
                    st = ctx.last_fit_stats()
                    print(json.dumps({"kind": "pca_sweep", "m": m, "s": s_out, "tol": tol,
                                      "max": c.max, "mean": c.mean,
                                      "pca_iterations": st["pca_iterations"], "pca_ms": st["pca_ms"],
                                      "fit_ms": st["total_ms"]}))
            for eps in a.eps:
                for tol in a.pca_sweep:
                    t0 = time.perf_counter()
                    A, m, s_out, c, rc = ctx.fit(X, eps=eps, m_cap=d, seed=11,
                                                 precision=lib.PREC_FP16X3, tol=tol)
                    torch.cuda.synchronize()
                    st = ctx.last_fit_stats()
                    print(json.dumps({"kind": "pca_sweep_dims", "eps": eps, "tol": tol, "m": m,
                                      "status": rc, "max": c.max, "probes": st["probes"],
                                      "pca_iterations": st["pca_iterations"], "pca_ms": st["pca_ms"],
                                      "seconds": time.perf_counter() - t0}))
            return
        for mode, s in MODES.items():
            for eps in a.eps:
                t0 = time.perf_counter()
                A, m, s_out, c, rc = ctx.fit(X, eps=eps, m_cap=d, s=d if s is None else s, seed=11,
                                             precision=lib.PREC_FP16X3, tol=a.tol)
                torch.cuda.synchronize()
                st = ctx.last_fit_stats()
                print(json.dumps({"kind": "dims_needed", "mode": mode, "eps": eps, "m": m,
                                  "s": s_out, "status": rc, "max": c.max, "mean": c.mean,
                                  "probes": st["probes"], "seconds": time.perf_counter() - t0}))
            for m in a.dims:
                if m > d:
                    continue
                ss = {"adagio": m // 2, "pca": m, "jl": 0}[mode]
                A, mm, s_out, c, rc = ctx.fit(X, eps=0.0, m=m, s=ss, seed=11,
                                              precision=lib.PREC_FP16X3, tol=a.tol)
                print(json.dumps({"kind": "distortion_at", "mode": mode, "m": m, "s": s_out,
                                  "max": c.max, "mean": c.mean, "violations_0.1": c.violations,
                                  "pairs": c.pairs}))


if __name__ == "__main__":
    main()
