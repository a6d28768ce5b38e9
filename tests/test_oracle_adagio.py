"""Pins for the oracle's JL matrix, Algorithm 1's map and the certified search.

* SplitMix64: the generator's published test values (tests/golden).
* Lemma 2 / Achlioptas: at the constructive k, all pairs keep their squared
  distance within (1 +- eps) with probability >= 1 - 1/n.
* Algorithm 1: data inside an s-dim affine subspace is embedded with zero
  distortion for every k (the JL part sees only Q(x - y) = 0).
* Theorem 2: padding JL rows for factor eps brings PCA's distortion delta_P
  down to at most delta_P * eps.
* Sec. 4.1 split rule and the search procedure on a hand-made predicate.
"""
import math
import os

import numpy as np
import pytest

from oracle import adagio as O
from oracle.certificate import certificate
from paper_1609_05388_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_values():
    vals = []
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            if line.startswith("seed"):
                seed = int(line.split()[1])
                continue
            vals.append(int(line))
    got = O.splitmix64_stream(seed, np.arange(len(vals)))
    assert [int(v) for v in got] == vals


def test_jl_entries_and_prefix_property():
    S = O.jl_matrix(7, 40, 300)
    k = 40
    assert set(np.unique(S * math.sqrt(k))) == {-1.0, 1.0}
    # rows do not depend on k except for the scale
    S_small = O.jl_matrix(7, 10, 300)
    np.testing.assert_array_equal(S_small * math.sqrt(10), S[:10] * math.sqrt(k))
    # sign balance: 12000 fair coins, 6 sigma
    frac = np.mean(S > 0)
    assert abs(frac - 0.5) < 6 * 0.5 / math.sqrt(S.size)
    # different seeds differ
    assert np.mean(O.jl_matrix(8, 40, 300) == S) < 0.6


def test_gaussian_option_moments():
    S = O.jl_matrix(3, 200, 200, dist="gaussian") * math.sqrt(200)
    assert abs(S.mean()) < 6 / 200
    assert abs(S.var() - 1.0) < 6 * math.sqrt(2) / 200


def test_gaussian_option_matches_the_normal_law():
    """Kolmogorov-Smirnov distance of the scaled entries to the standard normal
    CDF (scipy's, an independent implementation), for the whole matrix and for
    single rows and columns: a wrong Box-Muller transform (a dropped factor of
    2, sin/cos of the wrong uniform, a missing sqrt) fails it."""
    stats = pytest.importorskip("scipy.stats")
    k, d = 100, 400
    S = O.jl_matrix(12345, k, d, dist="gaussian") * math.sqrt(k)
    assert stats.kstest(S.ravel(), "norm").pvalue > 1e-3
    assert stats.kstest(S[0], "norm").pvalue > 1e-4
    assert stats.kstest(S[:, 7], "norm").pvalue > 1e-4
    # the two halves of the matrix are uncorrelated (independent counters)
    r = np.corrcoef(S[: k // 2].ravel(), S[k // 2:].ravel())[0, 1]
    assert abs(r) < 6 / math.sqrt(S.size / 2)


def achlioptas_k(n, eps, beta=1.0):
    return math.ceil((4 + 2 * beta) * math.log(n) / (eps * eps / 2 - eps ** 3 / 3))


def test_jl_bound_at_achlioptas_k():
    """Lemma 2: all pairs within (1 +- eps) in squared norm, w.p. >= 1 - 1/n."""
    n, d, eps = 50, 512, 0.5
    k = achlioptas_k(n, eps)
    assert k < d
    rng = np.random.default_rng(21)
    X = rng.standard_normal((n, d))
    I, J = np.triu_indices(n, 1)
    V = X[I] - X[J]
    fails = 0
    for seed in range(20):
        S = O.jl_matrix(seed, k, d)
        r = np.sum((V @ S.T) ** 2, axis=1) / np.sum(V * V, axis=1)
        fails += int(np.any((r < 1 - eps) | (r > 1 + eps)))
    assert fails <= 3            # expected <= 20/n = 0.4


def test_jl_scale_error_detected():
    """A 1/k scale (instead of 1/sqrt(k)) would break the bound everywhere."""
    n, d, eps = 50, 512, 0.5
    k = achlioptas_k(n, eps)
    rng = np.random.default_rng(21)
    X = rng.standard_normal((n, d))
    S = O.jl_matrix(0, k, d) / math.sqrt(k)
    v = X[0] - X[1]
    assert np.sum((S @ v) ** 2) / np.sum(v * v) < 1 - eps


@pytest.mark.parametrize("k", [1, 5, 40])
def test_affine_subspace_has_zero_distortion(k):
    rng = np.random.default_rng(31)
    s = 6
    X = synth.affine_subspace(rng, 150, 48, s).astype(np.float64)
    f = O.fit(X, s + k, seed=5, s=s)
    Y = O.embed(f.A, X)
    c = certificate(X, Y, eps=1e-6, lo=0.0, hi=1e-3)
    assert c.max < 1e-9
    # the JL rows annihilate the principal subspace
    assert np.max(np.abs(f.A[s:] @ f.pca.P[:s].T)) < 1e-12


def test_missing_residual_projection_detected():
    """Without Q = I - P^T P, the same data would be distorted."""
    rng = np.random.default_rng(31)
    s, k = 6, 5
    X = synth.affine_subspace(rng, 150, 48, s).astype(np.float64)
    pr = O.pca(X, s)
    S = O.jl_matrix(5, k, 48)
    A_wrong = np.vstack([pr.P, S])
    c = certificate(X, O.embed(A_wrong, X), eps=0.01)
    assert c.max > 0.1


def test_theorem2_padding_reduces_distortion():
    n, d, s, eps = 30, 40, 4, 0.5
    rng = np.random.default_rng(41)
    X = rng.standard_normal((n, d)) * np.linspace(5, 0.5, d)[None, :]
    pr = O.pca(X, s)
    delta_p = certificate(X, O.embed(pr.P, X), eps=0.5, lo=0.0, hi=1.0).max
    # Lemma 2 at eps/8 (squared norms), so ||SQv|| is within (1 +- eps/8)||Qv||
    k = achlioptas_k(n, eps / 8)
    fails = 0
    for seed in range(4):
        f = O.fit(X, s + k, seed=seed, s=s, pca_result=pr)
        c = certificate(X, O.embed(f.A, X), eps=0.5, lo=0.0, hi=1.0)
        fails += int(c.max > delta_p * eps)
    assert fails <= 1


def test_split_rule():
    assert O.split_rule(20) == (10, 10)
    assert O.split_rule(21) == (10, 11)
    assert O.split_rule(1) == (0, 1)


def test_gallop_bisect_procedure():
    calls = []

    def ok_at(t):
        def ok(r):
            calls.append(r)
            return r >= t
        return ok

    assert O.gallop_bisect(ok_at(37), 200) == (37, True)
    assert calls[:3] == [16, 32, 64]
    assert O.gallop_bisect(ok_at(5), 200) == (5, True)
    assert O.gallop_bisect(ok_at(300), 200) == (200, False)
    assert O.gallop_bisect(ok_at(200), 200) == (200, True)
    assert O.probe_sequence_start(100) == [16, 32, 64, 100]


def test_search_returns_certified_dimension_small():
    rng = np.random.default_rng(51)
    X = rng.standard_normal((200, 24)) * np.linspace(5, 0.2, 24)[None, :]
    res = O.search(X, eps=0.3, m_cap=24, seed=1)
    assert res.certified
    assert res.cert.max <= 0.3
    assert res.A.shape == (res.r, 24)
    # every failing probe below r really failed
    for r, mx in res.probes:
        assert (mx <= 0.3) == (r >= res.r) or r > res.r or mx > 0.3


def test_table3_ordering_on_mnist_shaped_data():
    """Table 3's qualitative ordering on the MNIST-shaped stand-in.

    Table 3 (MNIST-800, delta = 0.2): ADAGIO 95-98 dims, PCA 205, JL 260.  The
    spread spectrum of MNIST-like data is what makes ADAGIO win; on exactly
    low-rank data PCA alone is optimal, so the pin uses the MNIST-shaped family.
    """
    X = synth.mnist_like(seed=1, n=300, d=784).X.astype(np.float64)
    dims = {m: O.search(X, eps=0.2, m_cap=784, seed=3, mode=m).r
            for m in ("adagio", "pca", "jl")}
    assert dims["adagio"] < dims["pca"] < dims["jl"]


def test_fixed_mode_search_pads_a_fixed_pca_part():
    """The "fixed" mode (Theorem 2's construction) keeps s_fixed principal rows
    for every probe r >= s_fixed, padded with r - s_fixed JL rows; for
    r < s_fixed all r rows are principal.  On data inside a 6-dimensional
    affine subspace with s_fixed = 6, every probe r >= 6 has zero distortion
    (the JL rows see only Q(x - y) = 0) and every probe r < 6 projects out a
    spanned direction (some pair keeps almost none of its length), so the
    procedure must return exactly r = 6 with s = 6 and k = 0."""
    rng = np.random.default_rng(41)
    X = synth.affine_subspace(rng, 300, 40, 6).astype(np.float64)
    res = O.search(X, eps=0.3, m_cap=40, seed=4, mode="fixed", s_fixed=6)
    assert res.certified and res.r == 6
    assert res.cert.max < 1e-6
    assert [r for r, mx in res.probes if mx <= 0.3] == [r for r, _ in res.probes if r >= 6]
    for r, mx in res.probes:
        assert (mx < 1e-6) if r >= 6 else (mx > 0.5)


def test_jl_prefix_maps_are_rescaled_prefixes():
    """The reading behind the multi-candidate certificate: the map with kc JL
    rows (entries +-1/sqrt(kc), Algorithm 1) is the k-row map's first kc JL
    rows times sqrt(k / kc), with the same PCA part, so its embedding is
    [Y_P | sqrt(k / kc) Y_J[:, :kc]] and its squared distances are
    |dP|^2 + (k / kc) |dJ[:kc]|^2 (checked on the certificate, which recomputes
    every distance from the embedded coordinates)."""
    X = synth.small(seed=2, n=300).X.astype(np.float64)
    s, k = 6, 128
    f = O.fit(X, s + k, 9, s=s)
    Y = O.embed(f.A, X)
    for kc in (64, 100, 128):
        Sk = O.jl_matrix(9, kc, X.shape[1])
        np.testing.assert_allclose(Sk, np.sqrt(k / kc) * f.S[:kc], rtol=1e-15, atol=0)
        fc = O.fit(X, s + kc, 9, s=s, pca_result=f.pca)
        Yc = O.embed(fc.A, X)
        cand = np.hstack([Y[:, :s], np.sqrt(k / kc) * Y[:, s:s + kc]])
        np.testing.assert_allclose(Yc, cand, rtol=1e-12, atol=1e-12)
        a = certificate(X, Yc, 0.3)
        b = certificate(X, cand, 0.3)
        assert a.violations == b.violations and abs(a.max - b.max) <= 1e-12
        # and the prefix map is not the unscaled prefix: that one shrinks the JL part
        unscaled = np.hstack([Y[:, :s], Y[:, s:s + kc]])
        if kc < k:
            assert certificate(X, unscaled, 0.3).mean > a.mean
