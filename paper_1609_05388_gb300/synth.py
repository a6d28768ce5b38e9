"""Seeded synthetic workloads shaped like the paper's datasets.

The paper evaluates on MNIST (60 000 x 784, an 800-point subset in Sec. 4.1), the
UCR time-series sets of Table 2 and a few UCI sets.  None of those datasets is
available here, so every workload is drawn from a seeded generator with the
shape, value range and spectral structure of the paper's workloads.  This module
holds only input generation: no step of the embedding, of PCA or of the
distortion check lives here, so both the CUDA path and the CPU oracle can take
their inputs from it.

Workloads (all float32, row-major, one point per row):

* ``small``      2000 x 64: rank-8 Gaussian subspace with singular values
                 10 * 0.7**i plus iid N(0, 0.05^2) noise; eps 0.2.
* ``mnist_like`` 60 000 x 784 in [0, 1]: 10 Gaussian clusters in a rank-50
                 subspace, shifted and ReLU-clipped to about 80 % zeros,
                 scaled, clipped and quantised to k/255 (MNIST pixel grid);
                 eps 0.1.
* ``batched``    64 instances, n log-uniform in [500, 20000], d in
                 {128, 256, 512, 1024}, power-law spectrum i**-alpha with alpha
                 uniform in [0.5, 2] in a random orthonormal basis, plus
                 N(0, 0.01^2) noise; eps in {0.1, 0.2, 0.3}.
* ``large``      200 000 x 2048, power-law spectrum 1/i, 5 % of coordinates get
                 Laplace(0, 1) outliers; eps 0.1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Workload:
    name: str
    X: np.ndarray          # (n, d) float32, C-contiguous
    eps: float
    m_cap: int             # largest target dimension the search may return
    seed: int

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]

    @property
    def pairs(self) -> int:
        n = self.n
        return n * (n - 1) // 2


def _orthonormal(rng: np.random.Generator, d: int, r: int) -> np.ndarray:
    """d x r matrix with orthonormal columns (QR of a Gaussian matrix)."""
    g = rng.standard_normal((d, r))
    q, rr = np.linalg.qr(g)
    # fix the QR sign ambiguity so the basis is a deterministic function of g
    q *= np.sign(np.diag(rr))[None, :]
    return q


def small(seed: int = 0, n: int = 2000, d: int = 64) -> Workload:
    """Rank-8 subspace, singular values 10*0.7**i, plus N(0, 0.05^2) noise."""
    rng = np.random.default_rng(seed)
    r = 8
    U = _orthonormal(rng, d, r)
    sig = 10.0 * 0.7 ** np.arange(r)
    z = rng.standard_normal((n, r))
    X = (z * sig[None, :]) @ U.T + 0.05 * rng.standard_normal((n, d))
    return Workload("small", np.ascontiguousarray(X, dtype=np.float32), 0.2, 32, seed)


def mnist_like(seed: int = 1, n: int = 60000, d: int = 784, rank: int = 50,
               clusters: int = 10, zero_frac: float = 0.8) -> Workload:
    """MNIST-shaped data: clustered rank-50 signal, ReLU to ~80 % zeros, k/255."""
    rng = np.random.default_rng(seed)
    U = _orthonormal(rng, d, rank)
    centres = rng.standard_normal((clusters, rank))
    labels = rng.integers(0, clusters, size=n)
    z = centres[labels] + 0.5 * rng.standard_normal((n, rank))
    t = z @ U.T                                        # (n, d), rank-50 signal
    shift = np.quantile(t, zero_frac)
    t = np.maximum(t - shift, 0.0)
    scale = np.quantile(t[t > 0], 0.999) if np.any(t > 0) else 1.0
    t = np.clip(t / scale, 0.0, 1.0)
    X = np.round(t * 255.0) / 255.0
    return Workload("mnist_like", np.ascontiguousarray(X, dtype=np.float32), 0.1, d, seed)


def power_law(rng: np.random.Generator, n: int, d: int, alpha: float,
              noise: float = 0.01) -> np.ndarray:
    """Coordinates ~ N(0, i**(-2 alpha)) in a random orthonormal basis, plus noise."""
    Q = _orthonormal(rng, d, d)
    sig = np.arange(1, d + 1, dtype=np.float64) ** (-alpha)
    z = rng.standard_normal((n, d)) * sig[None, :]
    X = z @ Q.T + noise * rng.standard_normal((n, d))
    return np.ascontiguousarray(X, dtype=np.float32)


def batched(seed: int = 2, count: int = 64, n_lo: int = 500, n_hi: int = 20000,
            dims=(128, 256, 512, 1024)) -> list[Workload]:
    """Ragged batch of power-law instances (uneven n and d)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(rng.choice(dims))
        alpha = float(rng.uniform(0.5, 2.0))
        eps = float(rng.choice([0.1, 0.2, 0.3]))
        X = power_law(rng, n, d, alpha)
        out.append(Workload(f"batched[{b}]", X, eps, d, seed))
    return out


def large(seed: int = 4, n: int = 200000, d: int = 2048, outlier_frac: float = 0.05,
          chunk: int = 20000) -> Workload:
    """Power-law spectrum 1/i plus 5 % Laplace(0, 1) outlier coordinates."""
    rng = np.random.default_rng(seed)
    Q = _orthonormal(rng, d, d).astype(np.float32)
    sig = (1.0 / np.arange(1, d + 1, dtype=np.float64)).astype(np.float32)
    X = np.empty((n, d), dtype=np.float32)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        z = rng.standard_normal((r1 - r0, d), dtype=np.float32) * sig[None, :]
        blk = z @ Q.T
        mask = rng.random((r1 - r0, d), dtype=np.float32) < outlier_frac
        blk += mask * rng.laplace(0.0, 1.0, size=(r1 - r0, d)).astype(np.float32)
        X[r0:r1] = blk
    return Workload("large", X, 0.1, d, seed)


def mnist_like_family(rng: np.random.Generator, n: int, d: int = 784) -> tuple[np.ndarray, float]:
    """One instance of the mnist_like family with varied rank, clusters and eps.

    Used to build the training set of the dimension predictor: n, the signal
    rank, the number of clusters and eps vary so that every input feature of the
    predictor varies across instances.
    """
    rank = int(rng.integers(10, 80))
    clusters = int(rng.integers(2, 20))
    zero_frac = float(rng.uniform(0.6, 0.9))
    eps = float(rng.choice([0.1, 0.15, 0.2, 0.3]))
    wl = mnist_like(seed=int(rng.integers(0, 2**31 - 1)), n=n, d=d, rank=rank,
                    clusters=clusters, zero_frac=zero_frac)
    return wl.X, eps


def affine_subspace(rng: np.random.Generator, n: int, d: int, s: int,
                    offset_scale: float = 3.0) -> np.ndarray:
    """Points lying exactly (up to float32 rounding) in an s-dim affine subspace."""
    U = _orthonormal(rng, d, s)
    z = rng.standard_normal((n, s)) * np.linspace(3.0, 1.0, s)[None, :]
    c = offset_scale * rng.standard_normal(d)
    return np.ascontiguousarray(z @ U.T + c[None, :], dtype=np.float32)


WORKLOADS = {
    "small": small,
    "mnist_like": mnist_like,
    "large": large,
}
