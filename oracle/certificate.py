"""Loader for the plain-C FP64 certificate (``oracle/cert.c``) -- test infrastructure.

``build()`` compiles ``cert.c`` with gcc into ``oracle/_build/liboracle_cert.so``;
``certificate()`` runs it.  See ``cert.c`` for the definitions (Eq. 2, Eq. 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cert.c")
_SRCS = [_SRC, os.path.join(_HERE, "knn.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_cert.so")
MAX_BINS = 256


class _Cert(ctypes.Structure):
    _fields_ = [
        ("pairs", ctypes.c_uint64),
        ("degenerate", ctypes.c_uint64),
        ("violations", ctypes.c_uint64),
        ("overflow", ctypes.c_uint64),
        ("hist", ctypes.c_uint64 * MAX_BINS),
        ("max", ctypes.c_double),
        ("argmax_i", ctypes.c_int64),
        ("argmax_j", ctypes.c_int64),
        ("sum", ctypes.c_double),
        ("sum_c", ctypes.c_double),
        ("near_edge", ctypes.c_uint64),
    ]


@dataclass
class OracleCert:
    pairs: int
    degenerate: int
    violations: int
    overflow: int
    hist: np.ndarray
    max: float
    argmax_i: int
    argmax_j: int
    sum: float
    eps: float
    lo: float
    hi: float
    near_edge: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def mean(self) -> float:
        good = self.pairs - self.degenerate
        return self.sum / good if good > 0 else 0.0


def build(force: bool = False) -> str:
    """Compile cert.c and knn.c (gcc, -O2, pthreads).  Returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # -ffp-contract=off keeps every FP64 operation individually rounded
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, *_SRCS, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_certificate.restype = ctypes.c_int
        lib.oracle_certificate.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int64,
            ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_Cert)]
        lib.oracle_certificate_tiles.restype = ctypes.c_int
        lib.oracle_certificate_tiles.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
            ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_Cert)]
        lib.oracle_knn.restype = ctypes.c_int
        lib.oracle_knn.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_pair_sqdist.restype = ctypes.c_int
        lib.oracle_pair_sqdist.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def certificate(X: np.ndarray, Y: np.ndarray, eps: float, lo: float = 0.0,
                hi: float | None = None, nbins: int = 64, rows=None,
                threads: int | None = None, edge_tol: float = 1e-6) -> OracleCert:
    """FP64 all-pairs certificate of the map row i of X -> row i of Y.

    Inputs are widened to float64 (exact for float32 data).

    ``hi`` defaults to 2*eps (64 uniform bins on [0, 2 eps)).  ``rows=(a, b)``
    restricts to pairs (i, j) with a <= i < b, i < j.  ``near_edge`` counts the
    pairs whose distortion lies within ``edge_tol`` of a bin edge or of eps (the
    pairs a faithful implementation may bin either way).
    """
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    if X.shape[0] != Y.shape[0]:
        raise ValueError("X and Y must have the same number of rows")
    if hi is None:
        hi = 2.0 * eps
    n, d = X.shape
    m = Y.shape[1]
    a, b = (0, n) if rows is None else rows
    res = _Cert()
    rc = _load().oracle_certificate(
        X.ctypes.data, d, Y.ctypes.data, m, n, d, m, float(eps), float(lo),
        float(hi), nbins, a, b, threads or default_threads(), float(edge_tol), ctypes.byref(res))
    if rc != 0:
        raise ValueError("oracle_certificate: bad arguments")
    return OracleCert(int(res.pairs), int(res.degenerate), int(res.violations),
                      int(res.overflow), np.array(res.hist[:nbins], dtype=np.int64),
                      float(res.max), int(res.argmax_i), int(res.argmax_j),
                      float(res.sum), float(eps), float(lo), float(hi), int(res.near_edge))


def certificate_tiles(X: np.ndarray, Y: np.ndarray, eps: float, t0: int, t1: int,
                      tile: int = 128, blocks: int = 0, lo: float = 0.0,
                      hi: float | None = None, nbins: int = 64, threads: int | None = None,
                      edge_tol: float = 1e-6) -> OracleCert:
    """The certificate over the pairs of tiles [t0, t1) of the upper triangle of
    tile x tile blocks, numbered row by row over ``blocks`` block rows (0:
    ceil(n / tile)) (``cert.c``): the pair set of one shard of the GPU
    library's sharded certificate."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    if X.shape[0] != Y.shape[0]:
        raise ValueError("X and Y must have the same number of rows")
    if hi is None:
        hi = 2.0 * eps
    n, d = X.shape
    m = Y.shape[1]
    res = _Cert()
    rc = _load().oracle_certificate_tiles(
        X.ctypes.data, d, Y.ctypes.data, m, n, d, m, float(eps), float(lo), float(hi), nbins,
        tile, blocks, t0, t1, threads or default_threads(), float(edge_tol), ctypes.byref(res))
    if rc != 0:
        raise ValueError("oracle_certificate_tiles: bad arguments")
    return OracleCert(int(res.pairs), int(res.degenerate), int(res.violations),
                      int(res.overflow), np.array(res.hist[:nbins], dtype=np.int64),
                      float(res.max), int(res.argmax_i), int(res.argmax_j),
                      float(res.sum), float(eps), float(lo), float(hi), int(res.near_edge))


def pair_sqdist(X: np.ndarray, Y: np.ndarray, I, J):
    """FP64 squared distances of listed pairs, by direct coordinate differences."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    dx2 = np.empty(I.shape[0], dtype=np.float64)
    dy2 = np.empty(I.shape[0], dtype=np.float64)
    rc = _load().oracle_pair_sqdist(X.ctypes.data, X.shape[1], Y.ctypes.data,
                                    Y.shape[1], X.shape[1], Y.shape[1],
                                    I.ctypes.data, J.ctypes.data, I.shape[0],
                                    dx2.ctypes.data, dy2.ctypes.data, default_threads())
    if rc != 0:
        raise ValueError("oracle_pair_sqdist: bad arguments")
    return dx2, dy2


def pair_distortion(X, Y, I, J):
    """Eq. 2 for listed pairs (NaN for a degenerate pair)."""
    dx2, dy2 = pair_sqdist(X, Y, I, J)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.abs(np.sqrt(dy2 / dx2) - 1.0)
