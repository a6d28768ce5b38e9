"""Times the dimension predictor on a batch of feature vectors.

    python -m paper_1609_05388_gb300.profile_mlp [--batch 4096] [--reps 200]

Feature vectors, outputs and targets stay on the device.  Per call of
adagio_mlp_forward, adagio_predict_m and adagio_mlp_train_step (forward,
backward and Adam on the batch) it prints the wall time (the calls that return
a host value synchronise) and, for the forward, the device time from CUDA
events.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import time

import torch

from . import adagio as lib


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=200)
    a = ap.parse_args()
    g = torch.Generator(device="cuda").manual_seed(0)
    feats = torch.randn(a.batch, 68, device="cuda", generator=g)
    target = torch.rand(a.batch, device="cuda", generator=g)
    y = torch.empty(a.batch, device="cuda")
    mi = torch.empty(a.batch, dtype=torch.int32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = {"batch": a.batch, "reps": a.reps}
    with lib.Context(0) as ctx:
        ctx.mlp_load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "predictor_mnist_like.bin"))
        fwd = lambda: ctx._check(lib.LIB.adagio_mlp_forward(ctx.h, feats.data_ptr(), a.batch,
                                                            y.data_ptr(), st))
        pred = lambda: ctx._check(lib.LIB.adagio_predict_m(ctx.h, feats.data_ptr(), a.batch,
                                                           mi.data_ptr(), st))
        loss = ctypes.c_double(0.0)
        train = lambda: ctx._check(lib.LIB.adagio_mlp_train_step(ctx.h, feats.data_ptr(),
                                                                 target.data_ptr(), a.batch, 1e-4,
                                                                 ctypes.byref(loss), st))
        for name, fn in (("forward", fwd), ("predict_m", pred), ("train_step", train)):
            for _ in range(10):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record()
            for _ in range(a.reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            out[name + "_us_wall"] = (time.perf_counter() - t0) / a.reps * 1e6
            out[name + "_us_device"] = e0.elapsed_time(e1) / a.reps * 1e3
    print(json.dumps(out))


if __name__ == "__main__":
    main()
