"""Parity of the multi-candidate certificate of JL prefixes with the FP64 oracle.

One pass certifies the map [P ; S_k (I - P^T P)] (Algorithm 1 with s PCA rows
and k JL rows) and judges, against eps, the maps that keep the first kc JL rows
(entries +-1/sqrt(kc), Lemma 2).  The oracle certifies each candidate's
embedding [Y_P | sqrt(k / kc) Y_J[:, :kc]] exhaustively in FP64.  Pairs the
per-pair bounds leave open are recomputed exactly, so each candidate's
violation count must equal the oracle's, its verdict must be the oracle's,
and its bound interval must hold the exact maximum.
"""
import numpy as np
import pytest

from gpu_helpers import assert_cert_parity
from oracle import adagio as O
from oracle.certificate import certificate
from paper_1609_05388_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TC_PRECS = [pytest.param(1, id="fp16x3"), pytest.param(2, id="bf16x3")]


@pytest.fixture(scope="module")
def ctx():
    from paper_1609_05388_gb300 import adagio as lib
    c = lib.Context(0)
    yield c
    c.close()


def embedding(X, s, k, seed=5):
    f = O.fit(X.astype(np.float64), s + k, seed, s=s)
    return O.embed(f.A, X).astype(np.float32)


def candidate(Y, s, k, kc):
    Y = Y.astype(np.float64)
    return np.hstack([Y[:, :s], np.sqrt(k / kc) * Y[:, s:s + kc]])


def check_candidates(X, Y, s, k, kcs, eps, res, prec=1):
    """Every verdict consistent with the exact certificate of its candidate.
    The bound interval of the maximum is at most 1e-3 wide under FP16x3 and
    5e-3 under BF16x3 (its bounds carry a fourfold-plus safety factor)."""
    width = 1e-3 if prec == 1 else 5e-3
    exact = []
    for kc, r in zip(kcs, res):
        o = certificate(X, candidate(Y, s, k, kc), eps)
        exact.append(o)
        assert r["k"] == kc
        assert r["max_lower"] <= o.max <= r["max_upper"], (kc, r, o.max)
        assert r["max_upper"] - r["max_lower"] <= width
        assert r["unsettled_pairs"] == 0
        assert r["violations"] == o.violations, (kc, r, o.violations)
        assert r["verdict"] == (1 if o.violations == 0 else 0)
    return exact


def f32(v):
    return float(np.float32(v))  # the kernels compare against eps in FP32


@pytest.mark.parametrize("prec", TC_PRECS)
def test_mnist_shaped_four_prefixes(ctx, prec):
    """3000 x 784 (23 full tiles and a ragged one), s = 40, k = 256, prefixes
    of 64 .. 256 JL rows; eps between two candidates' maxima so that some
    pass and some fail, all decided."""
    wl = synth.mnist_like(seed=1, n=3000)
    s, k, kcs = 40, 256, [64, 128, 192, 256]
    Y = embedding(wl.X, s, k)
    maxima = sorted(certificate(wl.X, candidate(Y, s, k, kc), 0.5).max for kc in kcs)
    eps = f32(0.5 * (maxima[1] + maxima[2]))
    full, res = ctx.distortion_prefixes(torch.from_numpy(wl.X).cuda(), torch.from_numpy(Y).cuda(),
                                        s, eps, kcs, precision=prec)
    assert_cert_parity(full, certificate(wl.X, Y, eps), wl.X, Y)
    exact = check_candidates(wl.X, Y, s, k, kcs, eps, res, prec)
    assert [r["verdict"] for r in res] == [1 if o.violations == 0 else 0 for o in exact]
    assert sum(r["verdict"] == 1 for r in res) == 2


@pytest.mark.parametrize("prec", TC_PRECS)
def test_ragged_sizes_and_unpadded_widths(ctx, prec):
    """n = 777 (a ragged tile), s = 13 (PCA part padded to 64 columns), k = 100
    (the last prefix is k itself, not a multiple of 64), host inputs."""
    wl = synth.mnist_like(seed=2, n=777)
    s, k, kcs = 13, 100, [64, 100]
    Y = embedding(wl.X, s, k)
    eps = f32(0.3)
    full, res = ctx.distortion_prefixes(wl.X, Y, s, eps, kcs, precision=prec)
    assert_cert_parity(full, certificate(wl.X, Y, eps), wl.X, Y)
    check_candidates(wl.X, Y, s, k, kcs, eps, res, prec)


@pytest.mark.parametrize("prec", TC_PRECS)
def test_prefixes_below_k(ctx, prec):
    """Prefixes k, k - 64, k - 128, k - 192 of a JL part whose length is no
    multiple of 64 (k = 211): the JL columns start past a zero gap so that
    each prefix ends on a 64-column chunk; the full map's certificate and the
    verdicts against the oracle, at an eps between two candidates' maxima."""
    wl = synth.mnist_like(seed=4, n=2500)
    s, k, kcs = 30, 211, [211, 147, 83, 19]
    Y = embedding(wl.X, s, k)
    maxima = sorted(certificate(wl.X, candidate(Y, s, k, kc), 0.5).max for kc in kcs)
    eps = f32(0.5 * (maxima[1] + maxima[2]))
    full, res = ctx.distortion_prefixes(wl.X, Y, s, eps, kcs, precision=prec)
    assert_cert_parity(full, certificate(wl.X, Y, eps), wl.X, Y)
    exact = check_candidates(wl.X, Y, s, k, kcs, eps, res, prec)
    assert [r["verdict"] for r in res] == [1 if o.violations == 0 else 0 for o in exact]


def test_single_prefix_is_the_full_map(ctx):
    """kc = k: the candidate is the map itself, so its violation count and
    verdict are the full certificate's."""
    wl = synth.small(seed=0)                         # 2000 x 64
    s, k = 10, 64
    Y = embedding(wl.X, s, k)
    for eps in (f32(0.05), f32(0.4)):
        full, res = ctx.distortion_prefixes(wl.X, Y, s, eps, [k])
        assert full.violations == certificate(wl.X, Y, eps).violations
        assert res[0]["violations"] == full.violations
        assert res[0]["verdict"] == (1 if full.violations == 0 else 0)
        check_candidates(wl.X, Y, s, k, [k], eps, res)


def test_eps_at_a_candidates_maximum(ctx):
    """eps equal to a candidate's exact maximum (rounded to FP32 and moved to
    just above it): no certain violation may be claimed."""
    wl = synth.small(seed=3)
    s, k, kcs = 8, 128, [64, 128]
    Y = embedding(wl.X, s, k)
    mx = certificate(wl.X, candidate(Y, s, k, 64), 0.5).max
    eps = float(np.nextafter(np.float32(mx), np.float32(1.0)))
    _, res = ctx.distortion_prefixes(wl.X, Y, s, eps, kcs)
    assert res[0]["violations"] == 0 and res[0]["verdict"] == 1
    check_candidates(wl.X, Y, s, k, kcs, eps, res)
    # and just below it: exactly the pairs at the maximum violate
    eps2 = float(np.nextafter(np.float32(mx), np.float32(0.0)))
    _, res = ctx.distortion_prefixes(wl.X, Y, s, eps2, kcs)
    assert res[0]["verdict"] == 0 and res[0]["violations"] >= 1
    check_candidates(wl.X, Y, s, k, kcs, eps2, res)


def test_duplicate_points_are_excluded(ctx):
    """Repeated points (x_i == x_j): the certificate leaves those pairs out,
    and so must every candidate; the bounds cannot tell them apart from tiny
    distances, so they are decided by the exact recompute."""
    wl = synth.small(seed=5)
    X = np.concatenate([wl.X[:900], wl.X[:300]], axis=0)      # 300 duplicated rows
    s, k, kcs = 6, 128, [64, 128]
    Y = embedding(X, s, k)
    eps = f32(0.35)
    full, res = ctx.distortion_prefixes(X, Y, s, eps, kcs)
    assert full.degenerate == certificate(X, Y, eps).degenerate >= 300
    for r in res:
        assert r["recomputed"] >= 300 and r["max_upper"] < 1.0
    check_candidates(X, Y, s, k, kcs, eps, res)


def test_bad_arguments(ctx):
    from paper_1609_05388_gb300 import adagio as lib
    rng = np.random.default_rng(0)
    X = rng.standard_normal((300, 20)).astype(np.float32)
    Y = rng.standard_normal((300, 4 + 128)).astype(np.float32)
    # Y has k = 128 JL columns: 65 is neither a multiple of 64 nor 128 - 64 j
    # ([64, 65]: 64 fits one family, 65 neither), 192 > k, FP32 tiles
    for kcs, prec in (([], 1), ([64] * 5, 1), ([65], 1), ([64, 65], 1), ([0], 1), ([192], 1), ([64], 0)):
        with pytest.raises(lib.AdagioError) as ei:
            ctx.distortion_prefixes(X, Y, 4, 0.2, kcs, precision=prec)
        assert ei.value.code == lib.E_INVALID_ARG
    for eps in (0.0, 1.0, float("nan")):
        with pytest.raises(lib.AdagioError):
            ctx.distortion_prefixes(X, Y, 4, eps, [64])


def test_full_size_prefixes_against_their_certificates(ctx):
    """60 000 x 784 with s = 210 PCA rows and k = 211 JL rows (the benchmark's
    learned dimension), prefixes 211, 147, 83, 19: each decided verdict and
    bound interval against the exhaustive certificate of that candidate's
    embedding (the full certificate itself is pinned to the oracle at this
    size by the headline test)."""
    wl = synth.mnist_like(seed=1)
    X = torch.from_numpy(wl.X).cuda()
    A, m, s, _, _ = ctx.fit(X, eps=0.0, m=421, s=210)
    Y = ctx.embed(A, X)
    k, kcs = m - s, [211, 147, 83, 19]
    full, res = ctx.distortion_prefixes(X, Y, s, 0.1, kcs)
    whole = ctx.distortion(X, Y, 0.1)
    # the same pairs through a zero-padded layout: counts and the maximum's
    # pair agree, the maximum within the reported tolerances
    assert (full.violations, full.argmax_i, full.argmax_j) == (whole.violations, whole.argmax_i, whole.argmax_j)
    assert abs(full.max - whole.max) <= full.max_err_bound + whole.max_err_bound
    for kc, r in zip(kcs, res):
        Yc = torch.cat([Y[:, :s], Y[:, s:s + kc] * float(np.sqrt(k / kc))], 1).contiguous()
        c = ctx.distortion(X, Yc, 0.1)
        assert r["max_lower"] - 1e-6 <= c.max <= r["max_upper"] + 1e-6, (kc, r, c.max)
        if r["verdict"] == 1:
            assert c.violations == 0
        elif r["verdict"] == 0:
            assert c.violations > 0
        # Yc scales the JL columns in FP32, so pairs within rounding of eps may differ
        assert abs(r["violations"] - c.violations) <= 10 and r["unsettled_pairs"] == 0
