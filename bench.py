"""Benchmark: certified pairs/s and time-to-certified-embedding on the MNIST-shaped workload.

A step is one pass of the whole hot path over the 60 000 x 784 MNIST-shaped
input (eps = 0.1): centring, covariance and randomized PCA, JL matrix,
assembly, embedding, the learned dimension guess and its verification by the
exhaustive all-pairs certificate (the certified search continues from the
guess when it fails).  value = n(n-1)/2 / (step time): pairs of the returned
embedding certified per second of time-to-certified-embedding, inputs
resident in HBM.  Timed on the same input for comparison: the same split
precision with the plain search (no predictor), and the plain FP32 GPU path
(SIMT Gram tiles, plain search).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl adagio|reference]

N > 1 runs N independent replicas (one per GPU, launched by torchrun); the
certificate of one data set is not split across GPUs here.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

EPS = 0.1
# Residual tolerance of the randomized PCA (Sec. 4.5 uses randomized PCA as a
# stand-in for exact PCA; every returned map is certified exhaustively, so the
# tolerance only trades PCA time against how good the principal subspace is).
# At 1e-3 the block iteration stops after 7 iterations on this workload (the
# 4 to 7 power iterations of the randomized PCA the paper uses, Sec. 4.1) and
# the certified dimension stays within 1 % of the one at 1e-4 (24 iterations).
PCA_TOL = 1e-3
WORKLOAD = "mnist_like 60000x784 (10 clusters, rank-50, ~80% zeros, k/255), eps=0.1"
# The dimension the learned path returns on this workload (m = 428, s = 214,
# with the shipped predictor); the reference arm certifies the oracle's map of
# that dimension.
M_REF = 428
# Shards of the certificate whose first one the oracle recomputes to state the
# certificate's error (about 1.2e8 of the 1.8e9 pairs).
ORACLE_SHARDS = 15

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one tile-kernel
# launch on this workload (single-CTA tiles), by schedule band, each from one
# ncu capture of the full launch:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       --clock-control none -k regex:cert_tc_kernel -c 1
#       python -m paper_1609_05388_gb300.profile_cert --n 60000 --m 421 --reps 1
#       --tiles single --band B
# The traffic depends on the sizes and the schedule only.  A configuration
# without a capture (or a kernel changed since) reports null.
TRAFFIC_BYTES = {(1, 4): 15.42e9, (1, 8): 9.32e9, (1, 16): 7.49e9}


def workload_config():
    """The workload both arms measure (the same dictionary in both lines)."""
    return {"workload": WORKLOAD, "n": 60000, "d": 784, "eps": EPS,
            "pairs": 60000 * 59999 // 2, "pca_tol": PCA_TOL,
            "l2": "inputs larger than L2 (X 188 MB fp32; split planes 308 MB)"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="adagio", choices=["adagio", "reference"])
    p.add_argument("--precision", default="auto")
    p.add_argument("--no-cpu-baseline", action="store_true",
                   help="skip the oracle leg (its errors against the oracle and the CPU baseline)")
    p.add_argument("--no-legs", action="store_true",
                   help="skip the BF16x3, 200000 x 2048 and 64-instance batched legs")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-predictor", action="store_true",
                   help="time the plain search as the headline step")
    p.add_argument("--predictor", default="",
                   help="dimension predictor weights (default: the shipped MNIST-shaped one)")
    return p.parse_args()


PREDICTOR = os.path.join(ROOT, "paper_1609_05388_gb300", "predictor_mnist_like.bin")


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("gloo")
        pg = td
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, v):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz, sms=152):
    # 128 FP32 FMA lanes per SM, 2 flops per FMA
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def errors_vs_oracle(ctx, lib, X, X_host, A, m, s, prec):
    """Errors of the returned map and its certificate against the FP64 oracle
    (and the oracle's rate on the host cores, the CPU baseline).

    * Y = X A^T (Algorithm 1) on 4096 sampled rows against FP64 X A^T;
    * P = A[:s] (Sec. 2 PCA): orthonormality, and the energy it captures,
      tr(P C P^T), against the exact top-s eigenvalue sum of C = Xc^T Xc;
    * the JL part A[s:] against S (I - P^T P) with the oracle's S;
    * the certificate (Eq. 2, Eq. 3): shard 0 of ORACLE_SHARDS computed by the
      library against the oracle's certificate of the same tiles."""
    import torch
    from oracle import adagio as O
    from oracle.certificate import certificate_tiles, default_threads
    n, d = X_host.shape
    Y = ctx.embed(A, X)
    torch.cuda.synchronize()
    Yh = Y.cpu().numpy()
    Ah = A.cpu().numpy().astype(np.float64) if hasattr(A, "cpu") else np.asarray(A, np.float64)
    rows = np.random.default_rng(0).choice(n, 4096, replace=False)
    ref = X_host[rows].astype(np.float64) @ Ah.T
    y_err = float(np.max(np.linalg.norm(Yh[rows] - ref, axis=1) /
                         np.maximum(np.linalg.norm(ref, axis=1), 1e-30)))
    P = Ah[:s]
    orth = float(np.abs(P @ P.T - np.eye(s)).max())
    _, Xc = O.centre(X_host)
    C = O.covariance(Xc)
    del Xc
    theta = np.sort(np.linalg.eigvalsh(C))[::-1]
    deficit = float(1.0 - np.trace(P @ C @ P.T) / theta[:s].sum())
    Sm = O.jl_matrix(11, m - s, d)
    jl_err = float(np.abs(Ah[s:] - Sm @ (np.eye(d) - P.T @ P)).max())
    part = ctx.distortion_shard(X, Y, EPS, 0, ORACLE_SHARDS, precision=prec)
    B = 2 * (-(-n // 256))
    t1 = (B * (B + 1) // 2) // ORACLE_SHARDS
    t0 = time.time()
    o = certificate_tiles(X_host, Yh, EPS, 0, t1, blocks=B)
    el = time.time() - t0
    g_mean = part.sum / max(part.pairs - part.degenerate, 1)
    g_hist = np.array(part.hist[:], dtype=np.int64)
    err = {"embedding_max_rel_row_err": y_err,
           "pca_orthonormality_max_abs": orth,
           "pca_captured_energy_rel_deficit": deficit,
           "jl_rows_max_abs_err": jl_err,
           "certificate_sample": f"tiles [0,{t1}) of {B * (B + 1) // 2} (shard 0 of {ORACLE_SHARDS}): "
                                 f"{o.pairs} pairs",
           "pairs_equal": bool(part.pairs == o.pairs),
           "hist_abs_diff": int(np.abs(g_hist - o.hist).sum()),
           "violations_diff": int(part.violations) - o.violations,
           "overflow_diff": int(part.overflow) - o.overflow,
           "near_edge_pairs": o.near_edge,
           "max_abs_err": abs(part.max - o.max),
           "mean_abs_err": abs(g_mean - o.mean)}
    cpu = {"value": o.pairs / el, "unit": "pairs/s", "cores": default_threads(), "kind": "oracle",
           "sample": f"FP64 direct-difference certificate of {o.pairs} pairs (tiles [0,{t1}) of the "
                     f"returned map, m={m}), {el:.1f} s; excludes the oracle's exact PCA and search"}
    return err, cpu


def cert_leg(ctx, lib, X, Y, eps, precision, reps=2):
    """Tile-kernel time, recompute time and queue of one certificate of (X, Y)."""
    ctx.set_timing(True)
    tile, rec = [], []
    for _ in range(reps):
        c = ctx.distortion(X, Y, eps, precision=precision)
        st = ctx.last_cert_stats()
        tile.append(st["tile_ms"])
        rec.append(st["recompute_ms"])
    ctx.set_timing(False)
    return c, min(tile), min(rec), st["queued"]


def tensor_frac(pairs, d, m, tile_ms, peak):
    flops = pairs * 2.0 * (d + m)
    achieved = flops / (tile_ms / 1e3) / 1e12
    return achieved, achieved / peak


def knn_leg(ctx, Y, peak, k=30):
    """The k = 30 nearest-neighbour graph of the returned embedding (Sec. 4.7),
    exact: 60 000 queries against the same 60 000 points."""
    import torch
    ctx.knn(Y[:1024], k, B=Y)           # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    idx, _ = ctx.knn(Y, k)
    el = time.perf_counter() - t0
    n, m = Y.shape
    gram_flops = 2.0 * n * n * m
    return {"workload": f"k={k} nearest-neighbour graph of the embedding ({n} x {m})",
            "seconds": el, "queries_per_s": n / el,
            "gram_tflops": gram_flops / el / 1e12, "gram_frac_of_bf16_peak": gram_flops / el / 1e12 / peak,
            "rows_searched_exactly": ctx.knn_last_exact_rows()}


def prefix_leg(ctx, X, Y, s, m, eps, reps=2):
    """The multi-candidate certificate on the returned map: its own
    certificate plus the verdicts of the JL prefixes k, k - 64, k - 128,
    k - 192 in one pass, against one plain certificate of the map."""
    import torch
    k = m - s
    kcs = [kc for kc in (k, k - 64, k - 128, k - 192) if kc >= 1]
    ctx.set_timing(True)
    t_multi, t_one = [], []
    for _ in range(reps):
        full, res = ctx.distortion_prefixes(X, Y, s, eps, kcs)
        t_multi.append(ctx.last_cert_stats()["tile_ms"])
        ctx.distortion(X, Y, eps)
        t_one.append(ctx.last_cert_stats()["tile_ms"])
    ctx.set_timing(False)
    torch.cuda.synchronize()
    return {"workload": f"JL prefixes {kcs} of the returned map (s={s}, k={k}) in one pass",
            "tile_ms": min(t_multi), "tile_ms_plain_certificate": min(t_one),
            "full_max": full.max,
            "prefixes": [{"k": r["k"], "m": s + r["k"], "verdict": r["verdict"],
                          "max_interval": [r["max_lower"], r["max_upper"]],
                          "violations": r["violations"], "recomputed": r["recomputed"],
                          "unsettled_pairs": r["unsettled_pairs"]} for r in res]}


def large_leg(ctx, lib, peak, prec):
    """The 200 000 x 2048 workload (power-law spectrum, 5 % Laplace outliers):
    one exhaustive certificate (2.0e10 pairs) of a JL map of 300 rows."""
    import torch
    from paper_1609_05388_gb300 import synth
    wl = synth.large(seed=4)
    n, d, m = wl.X.shape[0], wl.X.shape[1], 300
    Xd = torch.from_numpy(wl.X).cuda()
    S = torch.from_numpy(ctx.jl_matrix(9, m, d)).cuda()
    Y = ctx.embed(S, Xd)
    c, tile_ms, rec_ms, q = cert_leg(ctx, lib, Xd, Y, 0.1, prec)
    pairs = n * (n - 1) // 2
    ach, frac = tensor_frac(pairs, d, m, tile_ms, peak)
    out = {"workload": "large 200000x2048 (power-law 1/i, 5% Laplace outliers), JL map m=300, eps=0.1",
           "pairs": pairs, "tile_ms": tile_ms, "recompute_ms": rec_ms, "queued": q,
           "certificate_pairs_per_s": pairs / ((tile_ms + rec_ms) / 1e3),
           "tile_pairs_per_s": pairs / (tile_ms / 1e3), "achieved_tflops": ach, "frac": frac,
           "max": c.max, "violations": c.violations}
    del Xd, Y
    torch.cuda.empty_cache()
    return out


def batched_leg(ctx, lib, prec):
    """The 64-instance ragged workload fitted and certified in one batched call
    (n log-uniform in [500, 20000], d in {128, ..., 1024}, eps in {0.1, 0.2, 0.3})."""
    import torch
    from paper_1609_05388_gb300 import synth
    wls = synth.batched()
    dX = [torch.from_numpy(w.X).cuda() for w in wls]
    epss = [w.eps for w in wls]
    ctx.fit_batched(dX[:2], epss[:2], precision=prec, graph=True)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = ctx.fit_batched(dX, epss, precision=prec, graph=True)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    pairs = sum(w.X.shape[0] * (w.X.shape[0] - 1) // 2 for w in wls)
    st = ctx.last_batch_stats()
    return {"workload": "batched: 64 instances, n log-uniform [500, 20000], d in {128,256,512,1024}, "
                        "power-law spectra, eps in {0.1,0.2,0.3}",
            "instances": len(wls), "pairs_per_certificate_set": pairs, "seconds": el,
            "certified": sum(1 for r in res if r["status"] == 0),
            "full_certificates": sum(r["full_certs"] for r in res),
            "probes": sum(r["probes"] for r in res),
            "rounds": st["rounds"], "graphs": st["graphs"],
            "certified_pairs_per_s": pairs / el}


def run_reference(args, rank, world, pg):
    """--impl reference: the FP64 CPU oracle as it stands, on the host cores.

    The oracle's own map of the workload (exact PCA of all 60 000 points,
    Algorithm 1 at m = M_REF, the same JL seed as the GPU fit) is certified
    by the oracle's direct-difference certificate, one bounded band of rows
    per step (every pair (i, j), j > i, of those rows)."""
    if rank != 0:
        return
    from paper_1609_05388_gb300 import synth
    from oracle.certificate import certificate, default_threads
    from oracle import adagio as O
    wl = synth.mnist_like(seed=1)
    X = wl.X
    f = O.fit(X.astype(np.float64), M_REF, 11)
    Y = O.embed(f.A, X)
    rows = 16
    for _ in range(args.warmup):
        certificate(X, Y, EPS, rows=(0, 1))
    times, pairs = [], 0
    for s in range(args.steps):
        t0 = time.time()
        c = certificate(X, Y, EPS, rows=(s * rows, (s + 1) * rows))
        times.append(time.time() - t0)
        pairs += c.pairs
    tot = sum(times)
    v = pairs / tot
    sample = (f"FP64 certificate of {rows} rows x all j>i per step of the oracle's map "
              f"(exact PCA of all {X.shape[0]} points, m={M_REF})")
    line = {"metric": "certified pairs/s", "value": v, "unit": "pairs/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "config": workload_config(),
            "cpu_baseline": {"kind": "oracle", "cores": default_threads(), "value": v,
                             "unit": "pairs/s", "sample": sample},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local, pg = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world, pg)
        return
    import torch
    from paper_1609_05388_gb300 import adagio as lib
    from paper_1609_05388_gb300 import synth

    torch.cuda.set_device(local)
    prec = {"auto": lib.PREC_FP16X3, "fp32": lib.PREC_FP32, "fp16x3": lib.PREC_FP16X3,
            "bf16x3": lib.PREC_BF16X3}[args.precision]
    wl = synth.mnist_like(seed=1)
    X_host = wl.X
    n, d = X_host.shape
    pairs = n * (n - 1) // 2
    X = torch.from_numpy(X_host).cuda()
    ctx = lib.Context(local)
    st = torch.cuda.current_stream()

    learned = 0 if args.no_predictor else 1
    if learned:
        ctx.mlp_load(args.predictor or PREDICTOR)

    def step(precision, use_predictor=learned, Xin=X):
        return ctx.fit(Xin, eps=EPS, m_cap=d, seed=11, precision=precision,
                       use_predictor=use_predictor, tol=PCA_TOL)

    wres = None
    for _ in range(max(args.warmup, 1)):
        wres = step(prec)
    # untimed: the autotuner picks the tile configuration for this size class
    # on the warm-up fit's map; the timed steps certify with it
    tile_cfg = None
    if prec != lib.PREC_FP32:
        Yw = ctx.embed(wres[0], X)
        tile_cfg = ctx.autotune_tiles(X, Yw, EPS, precision=prec)
        del Yw
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = lib.launch_count()
    barrier(pg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    results = [step(prec) for _ in range(args.steps)]
    e1.record(st)
    torch.cuda.synchronize()
    barrier(pg)
    launches = lib.launch_count() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(pg, ms)
    A, m, s, cert, rc = results[-1]
    fit_stats = ctx.last_fit_stats()
    value = sum_over_ranks(pg, pairs / (ms / 1e3))

    def timed(precision, use_predictor):
        step(precision, use_predictor)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(st)
        pr = step(precision, use_predictor)
        f1.record(st)
        torch.cuda.synchronize()
        pms = f0.elapsed_time(f1)
        fs = ctx.last_fit_stats()
        return {"value": pairs / (pms / 1e3), "unit": "pairs/s", "ms_per_step": pms, "m": pr[1],
                "max": pr[3].max, "max_err_bound": pr[3].max_err_bound,
                "probes": fs["probes"], "full_certs": fs["full_certs"]}

    # the same precision with the plain search, and the plain FP32 GPU path
    # (SIMT tiles, plain search), on the same input
    plain_search = plain = None
    if not args.no_plain:
        if learned:
            plain_search = timed(prec, 0)
        if prec != lib.PREC_FP32:
            plain = timed(lib.PREC_FP32, 0)

    # roofline of the dominant kernel (the all-pairs tile kernel) at the returned m
    Y = ctx.embed(A, X)
    ctx.set_timing(True)
    tiles_ms = []
    for _ in range(3):
        c1 = ctx.distortion(X, Y, EPS, precision=prec)
        tiles_ms.append(ctx.last_cert_stats()["tile_ms"])
    cst = ctx.last_cert_stats()
    ctx.set_timing(False)
    tile_ms = statistics.mean(tiles_ms)
    flops = pairs * 2.0 * (d + m)
    peaks, peak_src = measured_peaks()
    if prec == lib.PREC_FP32:
        sm_mhz = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = fp32_alu_peak_tflops(sm_mhz)
        roof = {"bound": "alu", "peak_source": "FP32 FMA lanes x clock (derived)"}
    else:
        peak = peaks["bf16_tflops"]
        roof = {"bound": "tensor", "peak_source": f"bf16_tflops ({peak_src})"}
    achieved = flops / (tile_ms / 1e3) / 1e12
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": TRAFFIC_BYTES.get((tile_cfg["variant"], tile_cfg["band"])) if tile_cfg else None,
                 "kernel_ms": tile_ms,
                 "algorithmic_flops_per_launch": flops,
                 "queued_pairs": cst["queued"]})
    if prec != lib.PREC_FP32:
        # tensor-pipe work actually issued: three products per K term over
        # the padded K (multiples of 64) and the full 128 x 128 tiles
        T = -(-n // 256) * 2
        tiles = T * (T + 1) // 2
        kpad = -(-d // 64) * 64 + -(-m // 64) * 64
        executed = tiles * 128 * 128 * 2.0 * kpad * 3
        roof["executed_tflops"] = executed / (tile_ms / 1e3) / 1e12
        roof["executed_frac"] = roof["executed_tflops"] / peak
        roof["tile_kernel"] = {1: "single CTA per 128x128 tile", 2: "CTA pair per 256x128 tile"}[
            ctx.tile_kernel_for(n)]

    # end to end through the C ABI with host buffers (copies inside the call)
    torch.cuda.synchronize()
    # inputs and output in pinned host memory (allocated before the timed region)
    X_pin = torch.from_numpy(X_host).pin_memory()
    A_pin = torch.empty((d, d), dtype=torch.float32).pin_memory()
    t0 = time.perf_counter()
    ke = max(1, min(args.steps, 2))
    for _ in range(ke):
        Ah, mh, sh, ch, rch = ctx.fit(X_pin, eps=EPS, m_cap=d, seed=11, precision=prec,
                                      use_predictor=learned, A=A_pin, tol=PCA_TOL)
    e2e_s = (time.perf_counter() - t0) / ke
    e2e = {"value": sum_over_ranks(pg, pairs / e2e_s), "unit": "pairs/s",
           "h2d_bytes_per_step": int(X_host.nbytes), "d2h_bytes_per_step": int(mh * d * 4 + 712),
           "seconds_per_step": e2e_s}

    # errors against the FP64 oracle (and the oracle's own rate), then the
    # other workloads: BF16x3 tiles on this map, the 200 000 x 2048 workload,
    # the 64-instance batch
    cpu = err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        err, cpu = errors_vs_oracle(ctx, lib, X, X_host, A, m, s, prec)
    legs = None
    if rank == 0 and not args.no_legs and prec != lib.PREC_FP32:
        legs = {}
        cb, bt, br, bq = cert_leg(ctx, lib, X, Y, EPS, lib.PREC_BF16X3)
        ach, fr = tensor_frac(pairs, d, m, bt, peak)
        legs["bf16x3_same_map"] = {"tile_ms": bt, "recompute_ms": br, "queued": bq,
                                   "achieved_tflops": ach, "frac": fr, "max": cb.max,
                                   "certificate_pairs_per_s": pairs / ((bt + br) / 1e3)}
        legs["knn_graph_k30"] = knn_leg(ctx, Y, peak)
        legs["prefixes"] = prefix_leg(ctx, X, Y, s, m, EPS)
        del Y
        torch.cuda.empty_cache()
        legs["large_200000x2048"] = large_leg(ctx, lib, peak, prec)
        legs["batched_64"] = batched_leg(ctx, lib, prec)

    if rank == 0:
        line = {
            "metric": "certified pairs/s", "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {lib.PREC_FP32: "f32", lib.PREC_FP16X3: "f16x3", lib.PREC_BF16X3: "bf16x3"}[prec],
            "data": "synthetic",
            "config": workload_config(),
            "parallelism": "replicas" if world > 1 else "single-gpu",
            "search": ("learned guess verified by the exhaustive certificate, then "
                       "doubling and bisection from it on failure" if learned else
                       "doubling 16,32,64,... then bisection") +
                      "; failing probes stop at the first certain violation",
            "tile_config": tile_cfg,
            "predictor": os.path.basename(args.predictor or PREDICTOR) if learned else None,
            "time_to_certified_embedding_s": ms / 1e3,
            "result": {"m": m, "s": s, "max": cert.max, "mean": cert.mean,
                       "violations": cert.violations, "recomputed": cert.recomputed,
                       "max_err_bound": cert.max_err_bound, "err_vs_oracle": err},
            "fit_stats": fit_stats,
            "certificate_only": {"value": pairs / (tile_ms / 1e3), "unit": "pairs/s (tile kernel)"},
            "plain_search": plain_search,
            "plain_fp32": plain,
            "roofline": roof,
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "legs": legs,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
