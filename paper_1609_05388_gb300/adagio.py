"""Thin Python binding of the C ABI in include/adagio.h (argument marshalling only).

Arrays may be CUDA ``torch.Tensor``s (device path: the work is enqueued on the
current torch stream), or host arrays (numpy or CPU tensors: the library copies
them to the device and back inside the call).  Every computation runs in
``libadagio.so``; if the library is missing this module raises on import.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libadagio.so")

OK = 0
E_INVALID_ARG = -1
E_NONFINITE = -2
E_CUDA = -3
E_WORKSPACE = -4
E_QUEUE_OVERFLOW = -5
E_TIMEOUT = -6
E_NOT_CERTIFIABLE = -7
E_UNSUPPORTED = -8

PREC_FP32 = 0
PREC_FP16X3 = 1
PREC_BF16X3 = 2
# tile kernels of the split-precision certificate (adagio_set_tile_kernel)
TILES_AUTO = 0
TILES_SINGLE = 1
TILES_PAIR = 2
JL_RADEMACHER = 0
JL_GAUSSIAN = 1
HIST_BINS = 64

STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "NONFINITE", -3: "CUDA", -4: "WORKSPACE",
                -5: "QUEUE_OVERFLOW", -6: "TIMEOUT", -7: "NOT_CERTIFIABLE", -8: "UNSUPPORTED"}


class CertStruct(ctypes.Structure):
    _fields_ = [
        ("pairs", ctypes.c_uint64), ("degenerate", ctypes.c_uint64),
        ("violations", ctypes.c_uint64), ("overflow", ctypes.c_uint64),
        ("recomputed", ctypes.c_uint64), ("hist", ctypes.c_uint64 * HIST_BINS),
        ("max", ctypes.c_double), ("mean", ctypes.c_double),
        ("max_err_bound", ctypes.c_double), ("mean_err_bound", ctypes.c_double),
        ("argmax_i", ctypes.c_int64), ("argmax_j", ctypes.c_int64),
        ("hist_lo", ctypes.c_double), ("hist_hi", ctypes.c_double), ("eps", ctypes.c_double),
    ]


class CertPartStruct(ctypes.Structure):
    """adagio_cert_part: one shard's raw sums (adagio_distortion_shard)."""
    _fields_ = [
        ("pairs", ctypes.c_uint64), ("degenerate", ctypes.c_uint64),
        ("violations", ctypes.c_uint64), ("overflow", ctypes.c_uint64),
        ("recomputed", ctypes.c_uint64), ("hist", ctypes.c_uint64 * HIST_BINS),
        ("sum", ctypes.c_double), ("bound_sum", ctypes.c_double),
        ("max", ctypes.c_double), ("max_bound", ctypes.c_double),
        ("argmax_i", ctypes.c_int64), ("argmax_j", ctypes.c_int64),
        ("hist_lo", ctypes.c_double), ("hist_hi", ctypes.c_double), ("eps", ctypes.c_double),
        ("shard", ctypes.c_int32), ("nshards", ctypes.c_int32),
    ]


class PrefixCertStruct(ctypes.Structure):
    """adagio_prefix_cert: the verdict of one JL prefix."""
    _fields_ = [
        ("k", ctypes.c_int32), ("verdict", ctypes.c_int32),
        ("violations", ctypes.c_uint64), ("unsettled_pairs", ctypes.c_uint64),
        ("recomputed", ctypes.c_uint64),
        ("max_lower", ctypes.c_double), ("max_upper", ctypes.c_double),
    ]


class FitOptsStruct(ctypes.Structure):
    _fields_ = [
        ("eps", ctypes.c_double), ("m", ctypes.c_int), ("s", ctypes.c_int),
        ("seed", ctypes.c_uint64), ("jl_dist", ctypes.c_int), ("precision", ctypes.c_int),
        ("use_predictor", ctypes.c_int), ("hist_lo", ctypes.c_double),
        ("hist_hi", ctypes.c_double), ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
        ("oversample", ctypes.c_int),
    ]


class CertStatsStruct(ctypes.Structure):
    _fields_ = [("prep_ms", ctypes.c_double), ("tile_ms", ctypes.c_double),
                ("recompute_ms", ctypes.c_double), ("queued", ctypes.c_uint64),
                ("grid", ctypes.c_int), ("tiles", ctypes.c_int64)]


class TileConfigStruct(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("band", ctypes.c_int), ("tile_ms", ctypes.c_double),
                ("size_class", ctypes.c_int)]


class FitStatsStruct(ctypes.Structure):
    _fields_ = [("probes", ctypes.c_int), ("full_certs", ctypes.c_int),
                ("pca_iterations", ctypes.c_int), ("s_computed", ctypes.c_int),
                ("pca_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("predicted_m", ctypes.c_int)]


class InstanceStruct(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int),
                ("ldx", ctypes.c_int64), ("eps", ctypes.c_double), ("m", ctypes.c_int),
                ("m_cap", ctypes.c_int), ("A", ctypes.c_void_p), ("m_out", ctypes.c_int),
                ("s_out", ctypes.c_int), ("status", ctypes.c_int), ("probes", ctypes.c_int),
                ("full_certs", ctypes.c_int), ("cert", CertStruct), ("feats", ctypes.c_void_p)]


class BatchStatsStruct(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int), ("graphs", ctypes.c_int), ("pca_rounds", ctypes.c_int),
                ("total_ms", ctypes.c_double)]


BATCH_GRAPH = 1


class AdagioError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"adagio error {code} ({STATUS_NAMES.get(code, '?')}): {msg}")
        self.code = code


@dataclass
class Certificate:
    pairs: int
    degenerate: int
    violations: int
    overflow: int
    recomputed: int
    hist: np.ndarray
    max: float
    mean: float
    max_err_bound: float
    mean_err_bound: float
    argmax_i: int
    argmax_j: int
    hist_lo: float
    hist_hi: float
    eps: float

    @classmethod
    def from_struct(cls, c: CertStruct) -> "Certificate":
        return cls(int(c.pairs), int(c.degenerate), int(c.violations), int(c.overflow),
                   int(c.recomputed), np.array(c.hist[:], dtype=np.int64), float(c.max),
                   float(c.mean), float(c.max_err_bound), float(c.mean_err_bound),
                   int(c.argmax_i), int(c.argmax_j), float(c.hist_lo), float(c.hist_hi),
                   float(c.eps))


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1609_05388_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "adagio_ctx_create": (i32, [i32, ctypes.c_size_t, ctypes.POINTER(vp)]),
        "adagio_ctx_destroy": (i32, [vp]),
        "adagio_last_error": (ctypes.c_char_p, [vp]),
        "adagio_workspace_bytes": (ctypes.c_size_t, [vp]),
        "adagio_default_fit_opts": (None, [ctypes.POINTER(FitOptsStruct)]),
        "adagio_distortion": (i32, [vp, vp, i64, i32, i64, vp, i32, i64, f64, f64, f64, i32,
                                    ctypes.POINTER(CertStruct), vp]),
        "adagio_embed": (i32, [vp, vp, i32, i32, i64, vp, i64, i64, vp, i64, vp]),
        "adagio_jl_matrix": (i32, [vp, ctypes.c_uint64, i32, i32, i32, vp, i64, vp]),
        "adagio_pca": (i32, [vp, vp, i64, i32, i64, i32, ctypes.POINTER(FitOptsStruct), vp, i64,
                             vp, vp]),
        "adagio_assemble": (i32, [vp, vp, i32, i64, vp, i32, i64, i32, vp, i64, vp]),
        "adagio_fit": (i32, [vp, vp, i64, i32, i64, ctypes.POINTER(FitOptsStruct), vp, i32,
                             ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(CertStruct),
                             vp]),
        "adagio_fit_batched": (i32, [vp, i32, ctypes.POINTER(InstanceStruct),
                                     ctypes.POINTER(FitOptsStruct), i32, vp]),
        "adagio_last_batch_stats": (i32, [vp, ctypes.POINTER(BatchStatsStruct)]),
        "adagio_set_timing": (i32, [vp, i32]),
        "adagio_set_tile_kernel": (i32, [vp, i32, i32]),
        "adagio_autotune_tiles": (i32, [vp, vp, i64, i32, i64, vp, i32, i64, f64, i32,
                                        ctypes.POINTER(TileConfigStruct), vp]),
        "adagio_tune_save": (i32, [vp, ctypes.c_char_p]),
        "adagio_tune_load": (i32, [vp, ctypes.c_char_p]),
        "adagio_tile_kernel_for": (i32, [vp, i64]),
        "adagio_last_cert_stats": (i32, [vp, ctypes.POINTER(CertStatsStruct)]),
        "adagio_launch_count": (ctypes.c_uint64, []),
        "adagio_last_fit_stats": (i32, [vp, ctypes.POINTER(FitStatsStruct)]),
        "adagio_mlp_num_params": (i64, []),
        "adagio_mlp_init": (i32, [vp, ctypes.c_uint64]),
        "adagio_mlp_set_params": (i32, [vp, vp, i64]),
        "adagio_mlp_get_params": (i32, [vp, vp, i64]),
        "adagio_mlp_forward": (i32, [vp, vp, i32, vp, vp]),
        "adagio_mlp_grad": (i32, [vp, vp, vp, i32, ctypes.POINTER(f64), vp, vp]),
        "adagio_mlp_train_step": (i32, [vp, vp, vp, i32, ctypes.c_float, ctypes.POINTER(f64), vp]),
        "adagio_predict_m": (i32, [vp, vp, i32, vp, vp]),
        "adagio_features": (i32, [vp, vp, i64, i32, i64, f64, ctypes.POINTER(FitOptsStruct), vp, vp]),
        "adagio_mlp_save": (i32, [vp, ctypes.c_char_p]),
        "adagio_mlp_load": (i32, [vp, ctypes.c_char_p]),
        "adagio_debug_tile_bounds": (i32, [vp, vp, i64, i32, i64, vp, i32, i64, i32, i64, i64, vp,
                                           vp, vp]),
        "adagio_distortion_noalloc": (i32, [vp, vp, i64, i32, i64, vp, i32, i64, f64, f64, f64,
                                            ctypes.POINTER(CertStruct), vp]),
        "adagio_distortion_shard": (i32, [vp, vp, i64, i32, i64, vp, i32, i64, f64, f64, f64, i32,
                                          i32, i32, ctypes.POINTER(CertPartStruct), vp]),
        "adagio_cert_merge": (i32, [ctypes.POINTER(CertPartStruct), i32, ctypes.POINTER(CertStruct)]),
        "adagio_knn": (i32, [vp, vp, i64, i64, vp, i64, i64, i32, i32, i32, vp, vp, vp]),
        "adagio_knn_last_exact_rows": (i64, [vp]),
        "adagio_distortion_prefixes": (i32, [vp, vp, i64, i32, i64, vp, i32, i32, i64, f64,
                                             ctypes.POINTER(i32), i32, i32,
                                             ctypes.POINTER(CertStruct),
                                             ctypes.POINTER(PrefixCertStruct), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def exported_symbols() -> list[str]:
    return [n for n in ("adagio_ctx_create", "adagio_ctx_destroy", "adagio_last_error",
                        "adagio_workspace_bytes", "adagio_default_fit_opts", "adagio_distortion",
                        "adagio_embed", "adagio_jl_matrix", "adagio_pca", "adagio_assemble",
                        "adagio_fit", "adagio_set_timing", "adagio_last_cert_stats",
                        "adagio_launch_count", "adagio_debug_tile_bounds",
                        "adagio_distortion_noalloc", "adagio_last_fit_stats",
                        "adagio_mlp_num_params", "adagio_mlp_init", "adagio_mlp_set_params",
                        "adagio_mlp_get_params", "adagio_mlp_forward", "adagio_mlp_grad",
                        "adagio_mlp_train_step", "adagio_predict_m", "adagio_features",
                        "adagio_mlp_save", "adagio_mlp_load", "adagio_fit_batched",
                        "adagio_last_batch_stats", "adagio_set_tile_kernel",
                        "adagio_tile_kernel_for", "adagio_autotune_tiles", "adagio_tune_save",
                        "adagio_tune_load", "adagio_distortion_shard", "adagio_cert_merge",
                        "adagio_knn", "adagio_knn_last_exact_rows",
                        "adagio_distortion_prefixes")
            if hasattr(LIB, n)]


def cert_merge(parts) -> "Certificate":
    """adagio_cert_merge of CertPartStruct parts (host only)."""
    arr = (CertPartStruct * len(parts))(*parts)
    c = CertStruct()
    rc = LIB.adagio_cert_merge(arr, len(parts), ctypes.byref(c))
    if rc != 0:
        raise AdagioError(rc, "adagio_cert_merge: parts are not shards 0..count-1 of one certificate")
    return Certificate.from_struct(c)


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(LIB.adagio_launch_count())


# ------------------------------------------------------------------ marshalling
class _Arr:
    """A 2-D float32 row-major array handed to the library (pointer + leading dim)."""

    def __init__(self, a, writable: bool = False):
        self.keep = a
        if _is_torch(a):
            import torch
            if a.dtype != torch.float32:
                raise TypeError("float32 tensors only")
            if a.dim() == 1:
                a = a.view(1, -1)
            if a.stride(1) != 1:
                raise ValueError("rows must be contiguous")
            if not a.is_cuda and not a.is_contiguous():
                raise ValueError("host tensors must be contiguous")
            self.keep = a
            self.ptr = a.data_ptr()
            self.rows, self.cols = a.shape
            self.ld = a.stride(0) if a.shape[0] > 1 else a.shape[1]
            self.cuda = a.is_cuda
        else:
            arr = np.asarray(a)
            if arr.dtype != np.float32 or not arr.flags.c_contiguous:
                if writable:
                    raise TypeError("output arrays must be C-contiguous float32")
                arr = np.ascontiguousarray(arr, dtype=np.float32)
            if arr.ndim == 1:
                arr = arr.reshape(1, -1)
            self.keep = arr
            self.ptr = arr.ctypes.data
            self.rows, self.cols = arr.shape
            self.ld = arr.shape[1]
            self.cuda = False


def _is_torch(a) -> bool:
    try:
        import torch
    except ImportError:
        return False
    return isinstance(a, torch.Tensor)


def _stream(*arrs) -> int:
    if any(getattr(a, "cuda", False) for a in arrs):
        import torch
        return torch.cuda.current_stream().cuda_stream
    return 0


class Context:
    """One library context on one CUDA device (owns the device workspace)."""

    def __init__(self, device: int = 0, workspace_limit: int = 0):
        h = ctypes.c_void_p()
        rc = LIB.adagio_ctx_create(device, workspace_limit, ctypes.byref(h))
        if rc != OK:
            raise AdagioError(rc, LIB.adagio_last_error(None).decode())
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            LIB.adagio_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int, allow=()):
        if rc != OK and rc not in allow:
            raise AdagioError(rc, LIB.adagio_last_error(self.h).decode())
        return rc

    @property
    def workspace_bytes(self) -> int:
        return int(LIB.adagio_workspace_bytes(self.h))

    def set_timing(self, enable: bool = True):
        self._check(LIB.adagio_set_timing(self.h, 1 if enable else 0))

    def set_tile_kernel(self, variant: int, band: int = 0):
        """Tile kernel of split-precision certificates (TILES_AUTO, TILES_SINGLE or TILES_PAIR)
        and the schedule's band height in tile rows (0: tuned or default)."""
        self._check(LIB.adagio_set_tile_kernel(self.h, int(variant), int(band)))

    def autotune_tiles(self, X, Y, eps: float, precision: int = PREC_FP16X3) -> dict:
        """Times every tile configuration on the certificate of (X, Y); the fastest is kept
        for n's size class.  Returns {variant, band, tile_ms, size_class}."""
        x, y = _Arr(X), _Arr(Y)
        if x.rows != y.rows:
            raise ValueError("X and Y must have the same number of rows")
        c = TileConfigStruct()
        self._check(LIB.adagio_autotune_tiles(self.h, x.ptr, x.rows, x.cols, x.ld, y.ptr, y.cols,
                                              y.ld, eps, precision, ctypes.byref(c), _stream(x, y)))
        return {"variant": c.variant, "band": c.band, "tile_ms": c.tile_ms,
                "size_class": c.size_class}

    def tune_save(self, path: str):
        self._check(LIB.adagio_tune_save(self.h, path.encode()))

    def tune_load(self, path: str):
        self._check(LIB.adagio_tune_load(self.h, path.encode()))

    def tile_kernel_for(self, n: int) -> int:
        """The tile kernel (TILES_SINGLE or TILES_PAIR) that certifies n points."""
        rc = LIB.adagio_tile_kernel_for(self.h, int(n))
        self._check(min(rc, 0))
        return rc

    def last_fit_stats(self) -> dict:
        st = FitStatsStruct()
        self._check(LIB.adagio_last_fit_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in FitStatsStruct._fields_}

    def last_cert_stats(self) -> dict:
        st = CertStatsStruct()
        self._check(LIB.adagio_last_cert_stats(self.h, ctypes.byref(st)))
        return {"prep_ms": st.prep_ms, "tile_ms": st.tile_ms, "recompute_ms": st.recompute_ms,
                "queued": int(st.queued), "grid": st.grid, "tiles": int(st.tiles)}

    # -------------------------------------------------------------- certificate
    def distortion(self, X, Y, eps: float, hist_lo: float = 0.0, hist_hi: float = 0.0,
                   precision: int = PREC_FP16X3) -> Certificate:
        x, y = _Arr(X), _Arr(Y)
        if x.rows != y.rows:
            raise ValueError("X and Y must have the same number of rows")
        c = CertStruct()
        self._check(LIB.adagio_distortion(self.h, x.ptr, x.rows, x.cols, x.ld, y.ptr, y.cols, y.ld,
                                          eps, hist_lo, hist_hi, precision, ctypes.byref(c),
                                          _stream(x, y)))
        return Certificate.from_struct(c)

    def distortion_shard(self, X, Y, eps: float, shard: int, nshards: int, hist_lo: float = 0.0,
                         hist_hi: float = 0.0, precision: int = PREC_FP16X3) -> CertPartStruct:
        x, y = _Arr(X), _Arr(Y)
        if x.rows != y.rows:
            raise ValueError("X and Y must have the same number of rows")
        part = CertPartStruct()
        self._check(LIB.adagio_distortion_shard(self.h, x.ptr, x.rows, x.cols, x.ld, y.ptr, y.cols,
                                                y.ld, eps, hist_lo, hist_hi, precision, shard,
                                                nshards, ctypes.byref(part), _stream(x, y)))
        return part

    def distortion_prefixes(self, X, Y, s: int, eps: float, kc,
                            precision: int = PREC_FP16X3):
        """(certificate of the whole map, [verdict dict per JL prefix]).

        Y = [PCA part (s columns) | k JL columns]; prefix c keeps kc[c] JL
        columns rescaled by sqrt(k / kc[c]).  verdict 1 = certified at eps,
        0 = violated (violations = the exact count), -1 = undecided."""
        x, y = _Arr(X), _Arr(Y)
        if x.rows != y.rows:
            raise ValueError("X and Y must have the same number of rows")
        kc = [int(v) for v in kc]
        ks = (ctypes.c_int * max(1, len(kc)))(*kc)
        outs = (PrefixCertStruct * max(1, len(kc)))()
        c = CertStruct()
        self._check(LIB.adagio_distortion_prefixes(self.h, x.ptr, x.rows, x.cols, x.ld, y.ptr, s,
                                                   y.cols - s, y.ld, eps, ks, len(kc), precision,
                                                   ctypes.byref(c), outs, _stream(x, y)))
        res = [{f: getattr(outs[i], f) for f, _ in PrefixCertStruct._fields_}
               for i in range(len(kc))]
        return Certificate.from_struct(c), res

    def debug_tile_bounds(self, X, Y, tiles: int, precision: int = PREC_FP16X3, stride: int = 1,
                          out=None):
        """(dump[tiles,128,128,4] = (dx2, dy2, ex, ey), tile_ij[tiles,2]) of the fast path,
        for every stride-th tile pair the tile kernel visits.  `out` may be a
        device tensor of that shape (float32) that receives the dump."""
        x, y = _Arr(X), _Arr(Y)
        if out is None:
            out = np.empty((tiles, 128, 128, 4), dtype=np.float32)
            optr = out.ctypes.data
        else:
            optr = out.data_ptr()
        ij = np.empty((tiles, 2), dtype=np.int32)
        self._check(LIB.adagio_debug_tile_bounds(self.h, x.ptr, x.rows, x.cols, x.ld, y.ptr, y.cols,
                                                 y.ld, precision, tiles, stride, optr,
                                                 ij.ctypes.data, _stream(x, y)))
        return out, ij

    def distortion_noalloc(self, X, Y, eps: float, hist_lo: float = 0.0,
                           hist_hi: float = 0.0) -> Certificate:
        """The certificate computed without any device allocation (small inputs, device arrays)."""
        x, y = _Arr(X), _Arr(Y)
        if x.rows != y.rows:
            raise ValueError("X and Y must have the same number of rows")
        c = CertStruct()
        self._check(LIB.adagio_distortion_noalloc(self.h, x.ptr, x.rows, x.cols, x.ld, y.ptr,
                                                  y.cols, y.ld, eps, hist_lo, hist_hi,
                                                  ctypes.byref(c), _stream(x, y)))
        return Certificate.from_struct(c)

    # ---------------------------------------------------------------- neighbours
    def knn(self, Q, k: int, B=None, exclude_self: bool | None = None):
        """The k nearest rows of B (default: Q itself, without each row's own
        index) for every row of Q: (idx int64 nq x k, d2 float64 nq x k),
        nearest first, ties by index.  Device arrays give device results."""
        q = _Arr(Q)
        b = q if B is None else _Arr(B)
        if exclude_self is None:
            exclude_self = B is None
        if q.cols != b.cols:
            raise ValueError("Q and B need the same number of columns")
        if q.cuda and b.cuda:
            import torch
            idx = torch.empty((q.rows, k), dtype=torch.int64, device=q.keep.device)
            d2 = torch.empty((q.rows, k), dtype=torch.float64, device=q.keep.device)
            pi, pd = idx.data_ptr(), d2.data_ptr()
        else:
            idx = np.empty((q.rows, k), dtype=np.int64)
            d2 = np.empty((q.rows, k), dtype=np.float64)
            pi, pd = idx.ctypes.data, d2.ctypes.data
        self._check(LIB.adagio_knn(self.h, q.ptr, q.rows, q.ld, b.ptr, b.rows, b.ld, q.cols, k,
                                   1 if exclude_self else 0, pi, pd, _stream(q, b)))
        return idx, d2

    def knn_last_exact_rows(self) -> int:
        return int(LIB.adagio_knn_last_exact_rows(self.h))

    # -------------------------------------------------------------------- embed
    def embed(self, A, X, Y=None):
        a, x = _Arr(A), _Arr(X)
        if Y is None:
            if x.cuda:
                import torch
                Y = torch.empty((x.rows, a.rows), dtype=torch.float32, device=x.keep.device)
            else:
                Y = np.empty((x.rows, a.rows), dtype=np.float32)
        y = _Arr(Y, writable=True)
        self._check(LIB.adagio_embed(self.h, a.ptr, a.rows, a.cols, a.ld, x.ptr, x.rows, x.ld,
                                     y.ptr, y.ld, _stream(a, x, y)))
        return Y

    # ---------------------------------------------------------------- fit steps
    def jl_matrix(self, seed: int, k: int, d: int, dist: int = JL_RADEMACHER, out=None):
        if out is None:
            out = np.empty((k, d), dtype=np.float32)
        o = _Arr(out, writable=True)
        self._check(LIB.adagio_jl_matrix(self.h, seed, k, d, dist, o.ptr, o.ld, _stream(o)))
        return out

    def pca(self, X, s: int, opts: FitOptsStruct | None = None, P=None):
        x = _Arr(X)
        if P is None:
            P = np.empty((s, x.cols), dtype=np.float32)
        p = _Arr(P, writable=True)
        theta = np.empty(s, dtype=np.float64)
        self._check(LIB.adagio_pca(self.h, x.ptr, x.rows, x.cols, x.ld, s,
                                   ctypes.byref(opts) if opts is not None else None, p.ptr, p.ld,
                                   theta.ctypes.data, _stream(x, p)))
        return P, theta

    def assemble(self, P, S, A=None):
        p = _Arr(P) if P is not None and np.size(P) else None
        s_ = _Arr(S) if S is not None and np.size(S) else None
        d = (p or s_).cols
        s, k = (p.rows if p else 0), (s_.rows if s_ else 0)
        if A is None:
            A = np.empty((s + k, d), dtype=np.float32)
        a = _Arr(A, writable=True)
        self._check(LIB.adagio_assemble(self.h, p.ptr if p else None, s, p.ld if p else d,
                                        s_.ptr if s_ else None, k, s_.ld if s_ else d, d, a.ptr,
                                        a.ld, _stream(a, *(v for v in (p, s_) if v))))
        return A

    # ------------------------------------------------------ dimension predictor
    @staticmethod
    def mlp_num_params() -> int:
        return int(LIB.adagio_mlp_num_params())

    def mlp_init(self, seed: int = 0):
        self._check(LIB.adagio_mlp_init(self.h, seed))

    def mlp_set_params(self, vec):
        v = np.ascontiguousarray(vec, dtype=np.float32)
        self._check(LIB.adagio_mlp_set_params(self.h, v.ctypes.data, v.size))

    def mlp_get_params(self) -> np.ndarray:
        v = np.empty(self.mlp_num_params(), dtype=np.float32)
        self._check(LIB.adagio_mlp_get_params(self.h, v.ctypes.data, v.size))
        return v

    def mlp_forward(self, feats) -> np.ndarray:
        f = np.ascontiguousarray(feats, dtype=np.float32).reshape(-1, 68)
        y = np.empty(f.shape[0], dtype=np.float32)
        self._check(LIB.adagio_mlp_forward(self.h, f.ctypes.data, f.shape[0], y.ctypes.data, None))
        return y

    def mlp_grad(self, feats, target):
        f = np.ascontiguousarray(feats, dtype=np.float32).reshape(-1, 68)
        t = np.ascontiguousarray(target, dtype=np.float32).reshape(-1)
        g = np.empty(self.mlp_num_params(), dtype=np.float32)
        loss = ctypes.c_double(0.0)
        self._check(LIB.adagio_mlp_grad(self.h, f.ctypes.data, t.ctypes.data, f.shape[0],
                                        ctypes.byref(loss), g.ctypes.data, None))
        return loss.value, g

    def mlp_train_step(self, feats, target, lr: float) -> float:
        f = np.ascontiguousarray(feats, dtype=np.float32).reshape(-1, 68)
        t = np.ascontiguousarray(target, dtype=np.float32).reshape(-1)
        loss = ctypes.c_double(0.0)
        self._check(LIB.adagio_mlp_train_step(self.h, f.ctypes.data, t.ctypes.data, f.shape[0],
                                              lr, ctypes.byref(loss), None))
        return loss.value

    def predict_m(self, feats) -> np.ndarray:
        f = np.ascontiguousarray(feats, dtype=np.float32).reshape(-1, 68)
        m = np.empty(f.shape[0], dtype=np.int32)
        self._check(LIB.adagio_predict_m(self.h, f.ctypes.data, f.shape[0], m.ctypes.data, None))
        return m

    def features(self, X, eps: float, opts: FitOptsStruct | None = None) -> np.ndarray:
        x = _Arr(X)
        out = np.empty(68, dtype=np.float32)
        self._check(LIB.adagio_features(self.h, x.ptr, x.rows, x.cols, x.ld, eps,
                                        ctypes.byref(opts) if opts is not None else None,
                                        out.ctypes.data, _stream(x)))
        return out

    def mlp_save(self, path: str):
        self._check(LIB.adagio_mlp_save(self.h, path.encode()))

    def mlp_load(self, path: str):
        self._check(LIB.adagio_mlp_load(self.h, path.encode()))

    # ---------------------------------------------------------------------- fit
    @staticmethod
    def default_opts(**kw) -> FitOptsStruct:
        o = FitOptsStruct()
        LIB.adagio_default_fit_opts(ctypes.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def fit(self, X, eps: float = 0.1, m: int = 0, m_cap: int | None = None, A=None,
            opts: FitOptsStruct | None = None, **kw):
        """Returns (A[:m], m, s, certificate, status)."""
        x = _Arr(X)
        o = opts if opts is not None else self.default_opts(eps=eps, m=m, **kw)
        if opts is None and eps <= 0:
            o.eps = 0.0
        if m_cap is None:
            m_cap = x.cols if o.eps > 0 else o.m
        if A is None:
            if x.cuda:
                import torch
                A = torch.empty((m_cap, x.cols), dtype=torch.float32, device=x.keep.device)
            else:
                A = np.empty((m_cap, x.cols), dtype=np.float32)
        a = _Arr(A, writable=True)
        mo, so = ctypes.c_int(0), ctypes.c_int(0)
        c = CertStruct()
        rc = self._check(LIB.adagio_fit(self.h, x.ptr, x.rows, x.cols, x.ld, ctypes.byref(o), a.ptr,
                                        m_cap, ctypes.byref(mo), ctypes.byref(so), ctypes.byref(c),
                                        _stream(x, a)), allow=(E_NOT_CERTIFIABLE,))
        return A[: mo.value], mo.value, so.value, Certificate.from_struct(c), rc

    def fit_batched(self, Xs, eps, m_cap=None, m=None, graph: bool = False,
                    features: bool = False, opts: FitOptsStruct | None = None, **kw):
        """Fits a list of CUDA float32 tensors (n_i x d_i) in one batched call.

        eps: one value or one per instance (<= 0: fixed m[i]).  Returns a list of
        dicts (A, m, s, status, probes, full_certs, cert, and with features=True
        the predictor's 68 features as a numpy array), A on the device.
        """
        import torch
        count = len(Xs)
        epss = list(eps) if hasattr(eps, "__len__") else [eps] * count
        caps = list(m_cap) if hasattr(m_cap, "__len__") else [m_cap] * count
        ms = list(m) if hasattr(m, "__len__") else [m] * count
        o = opts if opts is not None else self.default_opts(**kw)
        arr = (InstanceStruct * count)()
        keep = []
        for i, X in enumerate(Xs):
            if not (_is_torch(X) and X.is_cuda and X.dtype == torch.float32 and X.stride(1) == 1):
                raise TypeError("fit_batched takes CUDA float32 tensors with contiguous rows")
            n, d = X.shape
            cap = caps[i] if caps[i] is not None else (d if epss[i] > 0 else ms[i])
            A = torch.empty((max(cap, 1), d), dtype=torch.float32, device=X.device)
            keep.append((X, A))
            e = arr[i]
            e.X, e.n, e.d, e.ldx = X.data_ptr(), n, d, X.stride(0) if n > 1 else d
            e.eps = float(epss[i]) if epss[i] is not None else 0.0
            e.m = int(ms[i] or 0)
            e.m_cap = int(cap)
            e.A = A.data_ptr()
            if features:
                F = torch.zeros(68, dtype=torch.float32, device=X.device)
                keep[-1] = (X, A, F)
                e.feats = F.data_ptr()
        stream = torch.cuda.current_stream().cuda_stream
        self._check(LIB.adagio_fit_batched(self.h, count, arr, ctypes.byref(o),
                                           BATCH_GRAPH if graph else 0, stream))
        out = []
        for i in range(count):
            e = arr[i]
            out.append({"A": keep[i][1][: e.m_out], "m": e.m_out, "s": e.s_out,
                        "status": e.status, "probes": e.probes, "full_certs": e.full_certs,
                        "cert": Certificate.from_struct(e.cert)})
            if features:
                out[-1]["feats"] = keep[i][2].cpu().numpy()
        return out

    def last_batch_stats(self) -> dict:
        s = BatchStatsStruct()
        self._check(LIB.adagio_last_batch_stats(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in BatchStatsStruct._fields_}
