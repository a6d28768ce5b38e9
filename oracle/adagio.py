"""FP64 oracle of ADAGIO's fit, embedding and dimension search -- test infrastructure.

Every function follows a passage of the paper (arXiv 1609.05388) and is written
to be checked against it by eye; no blocking, fusion or reordering beyond the
definition.  Library primitives used as single steps: matrix products and the
symmetric eigendecomposition (LAPACK ``eigh``) of the covariance.

Readings of the paper taken here (ambiguous or garbled passages):
  * Sec. 2 "PCA" says PCA works on zero-centred data and projects on the
    leftmost columns of U in X = U Sigma V^T; with points as rows of X (n x d)
    the principal directions are the top eigenvectors of the d x d covariance
    Xc^T Xc (right singular vectors of the centred data).  P's rows are those
    eigenvectors, sorted by decreasing eigenvalue.
  * The map stays linear: f(w) = (Pw, S(w - P^T P w)) on the raw w (Algorithm 1);
    centring only chooses P.  Distances do not depend on it.
  * S has iid entries +-1/sqrt(k) (Algorithm 1, Lemma 2).  The random bits come
    from SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
    number generators", OOPSLA 2014) used as a counter: entry (i, j) takes the
    c-th output of the stream seeded with ``seed``, c = i*2^32 + 2j (+1 for the
    second uniform of the Gaussian option), sign = -1 when the top bit is set.
    Row i does not depend on k except for the 1/sqrt(k) scale.
  * Sec. 4.1: a target dimension r uses floor(r/2) principal components and
    ceil(r/2) JL rows.
  * Table 3's question "how many dimensions are needed for distortion delta" is
    answered by a certified search: probe r = 16, 32, 64, ... (capped) until the
    exhaustive certificate's maximum is <= eps, then bisect between the last
    failing and the first passing probe.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .certificate import OracleCert, certificate

# ---------------------------------------------------------------- SplitMix64
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_stream(seed: int, counters: np.ndarray) -> np.ndarray:
    """Output number ``c`` (0-based) of the SplitMix64 stream seeded with ``seed``.

    SplitMix64 advances its state by the golden-ratio increment and returns a
    mixed copy of it; output c therefore mixes seed + (c + 1) * gamma.
    """
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def jl_counters(k: int, d: int, second: bool = False) -> np.ndarray:
    i = np.arange(k, dtype=np.uint64)[:, None]
    j = np.arange(d, dtype=np.uint64)[None, :]
    return (i << np.uint64(32)) | (j << np.uint64(1)) | np.uint64(1 if second else 0)


def jl_matrix(seed: int, k: int, d: int, dist: str = "rademacher") -> np.ndarray:
    """S in R^{k x d} with iid entries +-1/sqrt(k) (Algorithm 1; Lemma 2).

    ``dist="gaussian"`` gives N(0, 1/k) entries by Box-Muller from two uniforms.
    """
    if k == 0:
        return np.zeros((0, d))
    z0 = splitmix64_stream(seed, jl_counters(k, d))
    if dist == "rademacher":
        sign = np.where((z0 >> np.uint64(63)) == np.uint64(1), -1.0, 1.0)
        return sign / math.sqrt(k)
    if dist == "gaussian":
        z1 = splitmix64_stream(seed, jl_counters(k, d, second=True))
        u1 = ((z0 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
        u2 = ((z1 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
        g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        return g / math.sqrt(k)
    raise ValueError(dist)


# ----------------------------------------------------------------------- PCA
def centre(X: np.ndarray):
    """Column mean and zero-centred copy (Sec. 2, PCA on zero-centred data)."""
    X64 = np.asarray(X, dtype=np.float64)
    mu = X64.mean(axis=0)
    return mu, X64 - mu[None, :]


def covariance(Xc: np.ndarray) -> np.ndarray:
    """C = Xc^T Xc (d x d), unnormalised; its eigenvectors are PCA's directions."""
    return Xc.T @ Xc


def canonical_signs(P: np.ndarray) -> np.ndarray:
    """Each row's entry of largest magnitude made positive (lowest index on ties)."""
    P = P.copy()
    for r in range(P.shape[0]):
        j = int(np.argmax(np.abs(P[r])))
        if P[r, j] < 0:
            P[r] = -P[r]
    return P


@dataclass
class PCAResult:
    P: np.ndarray        # (s, d) orthonormal rows, decreasing eigenvalue
    theta: np.ndarray    # all d eigenvalues of C, decreasing
    mu: np.ndarray       # column mean used for centring

    @property
    def sigma(self) -> np.ndarray:
        """Singular values of the centred data matrix."""
        return np.sqrt(np.maximum(self.theta, 0.0))


def pca(X: np.ndarray, s: int) -> PCAResult:
    """Top-s principal directions of X (Sec. 2 PCA; Algorithm 1's input P)."""
    mu, Xc = centre(X)
    C = covariance(Xc)
    w, V = np.linalg.eigh(C)                        # ascending eigenvalues
    order = np.lexsort((np.arange(w.size), -w))     # decreasing, ties by index
    w = w[order]
    V = V[:, order]
    P = canonical_signs(V[:, :s].T) if s > 0 else np.zeros((0, X.shape[1]))
    return PCAResult(P=P, theta=w, mu=mu)


# ---------------------------------------------------------------- Algorithm 1
def split_rule(r: int) -> tuple[int, int]:
    """Sec. 4.1: floor(r/2) principal components and ceil(r/2) JL rows."""
    s = r // 2
    return s, r - s


def assemble(P: np.ndarray, S: np.ndarray) -> np.ndarray:
    """A = [P ; S (I - P^T P)] so that A w = (P w, S(w - P^T P w)) (Algorithm 1)."""
    d = P.shape[1] if P.size else S.shape[1]
    Q = np.eye(d) - P.T @ P          # projector on the complement of P's rows
    return np.vstack([P, S @ Q])


def embed(A: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Row i of Y is f(x_i) = A x_i (the map of Algorithm 1 applied to every point)."""
    return np.asarray(X, dtype=np.float64) @ A.T


@dataclass
class FitResult:
    A: np.ndarray
    s: int
    k: int
    pca: PCAResult
    S: np.ndarray


def fit(X: np.ndarray, m: int, seed: int, s: int | None = None,
        dist: str = "rademacher", pca_result: PCAResult | None = None) -> FitResult:
    """ADAGIO map of target dimension m (Algorithm 1 with Sec. 4.1's split)."""
    if s is None:
        s, k = split_rule(m)
    else:
        k = m - s
    pr = pca_result if pca_result is not None else pca(X, s)
    P = pr.P[:s]
    S = jl_matrix(seed, k, X.shape[1], dist)
    return FitResult(A=assemble(P, S), s=s, k=k, pca=pr, S=S)


# ------------------------------------------------------------ certified search
@dataclass
class SearchResult:
    r: int
    certified: bool
    probes: list          # [(r, max distortion)]
    cert: OracleCert
    A: np.ndarray


def probe_sequence_start(cap: int) -> list[int]:
    seq, r = [], 16
    while r < cap:
        seq.append(r)
        r *= 2
    seq.append(cap)
    return seq


def gallop_bisect(ok, cap: int) -> tuple[int, bool]:
    """The certified-search procedure on a predicate ok(r).

    Probe r = 16, 32, 64, ... (the last probe is ``cap``) until ok(r); then
    bisect the interval (last failing probe, first passing probe] with
    mid = floor((lo + hi) / 2).  Returns (r, True) for the smallest passing
    probe met, or (cap, False) when even ``cap`` fails.
    """
    last_fail, first_ok = 0, None
    for r in probe_sequence_start(cap):
        if ok(r):
            first_ok = r
            break
        last_fail = r
    if first_ok is None:
        return cap, False
    lo, hi = last_fail, first_ok
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if ok(mid):
            hi = mid
        else:
            lo = mid
    return hi, True


def search(X: np.ndarray, eps: float, m_cap: int, seed: int,
           dist: str = "rademacher", threads: int | None = None,
           mode: str = "adagio", s_fixed: int = 0) -> SearchResult:
    """Smallest certified target dimension found by ``gallop_bisect``.

    ok(r) means the exhaustive certificate of the rank-r map has maximum
    distortion <= eps (Eq. 3).  ok is not guaranteed monotone in r (S is
    random), so the answer is the smallest passing probe this procedure meets.
    ``mode`` selects the map: "adagio" (Sec. 4.1 split), "pca" (r principal
    components only) or "jl" (r JL rows only), the three rows of Table 3
    this library can reproduce without NuMax; "fixed" is Theorem 2's
    construction: a PCA part of ``s_fixed`` rows (all r rows when r is
    smaller) padded with r - s_fixed JL rows on its residual.
    """
    d = X.shape[1]
    cap = min(m_cap, d)
    n_pc = {"pca": cap, "fixed": min(s_fixed, cap)}.get(mode, cap // 2)
    pr = pca(X, n_pc)
    probes = []
    cache = {}

    def ok(r):
        if r not in cache:
            s = {"adagio": r // 2, "pca": r, "jl": 0, "fixed": min(s_fixed, r)}[mode]
            f = fit(X, r, seed, s=s, dist=dist, pca_result=pr)
            Y = embed(f.A, X)
            c = certificate(X, Y, eps, threads=threads)
            cache[r] = (c.max <= eps, c, f.A)
            probes.append((r, c.max))
        return cache[r][0]

    r, certified = gallop_bisect(ok, cap)
    ok(r)
    _, c, A = cache[r]
    return SearchResult(r, certified, probes, c, A)
