"""k-nearest neighbours by brute force in FP64 -- test infrastructure.

The applications of Sec. 4.6 (10-nearest-neighbour vote on embedded SIFT
descriptors) and Sec. 4.7 (a k = 30 nearest-neighbour graph of the embedded
points) search the embedded space.  ``knn`` computes, for every query, the k
base points with the smallest Euclidean distance from coordinate differences in
FP64 (``knn.c``), ties broken by the smaller base index; ``exclude_self``
leaves point i out of query i's neighbours (the graph of one point set).
"""
from __future__ import annotations

import ctypes

import numpy as np

from .certificate import _load, default_threads


def knn(Q: np.ndarray, B: np.ndarray, k: int, exclude_self: bool = False,
        threads: int | None = None):
    """(idx (nq x k, int64), d2 (nq x k, float64)), nearest first."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if Q.shape[1] != B.shape[1]:
        raise ValueError("queries and base points need the same dimension")
    nq, m = Q.shape
    nb = B.shape[0]
    idx = np.empty((nq, k), dtype=np.int64)
    d2 = np.empty((nq, k), dtype=np.float64)
    rc = _load().oracle_knn(Q.ctypes.data, m, nq, B.ctypes.data, m, nb, m, k,
                            1 if exclude_self else 0, threads or default_threads(),
                            idx.ctypes.data, d2.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_knn: bad arguments")
    return idx, d2
