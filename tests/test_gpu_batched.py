"""The batched fit: every instance must get exactly what the single fit computes.

The single fit is parity-tested against the oracle elsewhere (JL rows
bit-exact, PCA subspace, search, certificate); here the batched call is held to
bit-identity with it on ragged batches, with and without graph capture, and
its search and maps are checked against the oracle on small instances.
"""
import numpy as np
import pytest

from gpu_helpers import assert_cert_parity
from oracle import adagio as O
from oracle.certificate import certificate
from paper_1609_05388_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1609_05388_gb300 import adagio as lib
    c = lib.Context(0)
    yield c
    c.close()


def _ragged(seed, count, n_lo, n_hi, dims):
    rng = np.random.default_rng(seed)
    Xs, epss = [], []
    for _ in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        d = int(rng.choice(dims))
        alpha = float(rng.uniform(0.5, 2.0))
        Xs.append(synth.power_law(rng, n, d, alpha))
        epss.append(float(rng.choice([0.1, 0.2, 0.3])))
    return Xs, epss


def _same_cert(a, b):
    assert a.pairs == b.pairs and a.degenerate == b.degenerate
    assert a.violations == b.violations and a.overflow == b.overflow
    assert np.array_equal(a.hist, b.hist)
    assert a.max == b.max and (a.argmax_i, a.argmax_j) == (b.argmax_i, b.argmax_j)
    assert a.mean == pytest.approx(b.mean, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("precision,graph", [(0, False), (1, False), (1, True), (2, True)])
def test_batched_equals_single_fits(ctx, precision, graph):
    Xs, epss = _ragged(5, 7, 200, 2500, (16, 48, 96, 130))
    # one fixed-dimension instance and one whose cap is too small to certify
    epss[2] = 0.0
    caps = [None] * len(Xs)
    ms = [None] * len(Xs)
    ms[2] = min(12, Xs[2].shape[1])
    caps[2] = ms[2]
    epss[4] = 0.05
    caps[4] = 4
    dX = [torch.from_numpy(X).cuda() for X in Xs]
    res = ctx.fit_batched(dX, epss, m_cap=caps, m=ms, graph=graph, precision=precision, seed=3)
    st = ctx.last_batch_stats()
    assert st["rounds"] >= 2 and (st["graphs"] == st["rounds"] if graph else st["graphs"] == 0)
    for i, X in enumerate(Xs):
        if epss[i] > 0:
            A, m, s, c, rc = ctx.fit(dX[i], eps=epss[i], m_cap=caps[i] or X.shape[1],
                                     precision=precision, seed=3)
        else:
            A, m, s, c, rc = ctx.fit(dX[i], eps=0.0, m=ms[i], m_cap=caps[i], precision=precision,
                                     seed=3)
        r = res[i]
        assert (r["m"], r["s"], r["status"]) == (m, s, rc), i
        assert torch.equal(r["A"], A), i
        _same_cert(r["cert"], c)
        if epss[i] > 0:
            fs = ctx.last_fit_stats()
            assert (r["probes"], r["full_certs"]) == (fs["probes"], fs["full_certs"]), i
    assert res[4]["status"] == -7 and res[4]["m"] == 4      # not certifiable at m_cap = 4


def test_batched_search_agrees_with_oracle(ctx):
    """Small instances: the oracle's search (exact PCA, same JL rows) reaches the
    same dimension up to probes whose verdict the oracle finds marginal, and the
    returned certificate is the exhaustive one of the returned map."""
    rng = np.random.default_rng(9)
    Xs = [synth.small(seed=s, n=n, d=d).X for s, n, d in ((0, 400, 32), (1, 700, 64), (2, 300, 48))]
    Xs.append(synth.affine_subspace(rng, 500, 40, 5))
    epss = [0.2, 0.2, 0.3, 0.1]
    caps = [32, 32, 48, 40]
    dX = [torch.from_numpy(X).cuda() for X in Xs]
    res = ctx.fit_batched(dX, epss, m_cap=caps, precision=1, seed=5)
    for X, eps, cap, r in zip(Xs, epss, caps, res):
        assert r["status"] == 0 and r["cert"].max <= eps
        ref = O.search(X.astype(np.float64), eps=eps, m_cap=cap, seed=5)
        assert ref.certified
        if r["m"] != ref.r:
            for rr, mx in ref.probes:
                if (rr < r["m"]) != (rr < ref.r):
                    assert abs(mx - eps) < 0.02, (r["m"], ref.r, ref.probes)
        Y = ctx.embed(r["A"].cpu().numpy(), X)
        c2 = ctx.distortion(X, Y, eps, precision=1)
        assert c2.max == r["cert"].max and np.array_equal(c2.hist, r["cert"].hist)


def test_batched_fixed_m_affine_subspace(ctx):
    """Data inside an affine s-dimensional subspace: the fixed-m map with s
    principal rows has zero distortion (Sec. 4.1), in every instance."""
    rng = np.random.default_rng(21)
    Xs = [synth.affine_subspace(rng, n, d, s) for n, d, s in ((900, 48, 6), (300, 20, 3), (1200, 64, 10))]
    ss = [6, 3, 10]
    dX = [torch.from_numpy(X).cuda() for X in Xs]
    for X, dx, s in zip(Xs, dX, ss):
        res = ctx.fit_batched([dx], [0.0], m=[s + 7], s=s, precision=0)
        assert res[0]["m"] == s + 7 and res[0]["s"] == s
        assert res[0]["cert"].max <= 2e-5
        ref = O.fit(X.astype(np.float64), s + 7, 0, s=s)
        np.testing.assert_allclose(res[0]["A"][s:].cpu().numpy(), ref.A[s:], atol=5e-4)


def test_batched_with_predictor_matches_single(ctx):
    Xs, epss = _ragged(13, 5, 300, 1500, (64, 100))
    ctx.mlp_init(7)          # an untrained network: guesses are poor, the search corrects them
    dX = [torch.from_numpy(X).cuda() for X in Xs]
    res = ctx.fit_batched(dX, epss, precision=1, seed=2, use_predictor=1)
    for i, X in enumerate(Xs):
        A, m, s, c, rc = ctx.fit(dX[i], eps=epss[i], precision=1, seed=2, use_predictor=1)
        assert (res[i]["m"], res[i]["s"], res[i]["status"]) == (m, s, rc), i
        assert torch.equal(res[i]["A"], A)
        assert (res[i]["cert"].max <= epss[i]) == (rc == 0)


def test_batched_rejects_nonfinite_and_bad_args(ctx):
    from paper_1609_05388_gb300 import adagio as lib
    Xs, epss = _ragged(17, 3, 100, 200, (8,))
    Xs[1][5, 3] = np.nan
    dX = [torch.from_numpy(X).cuda() for X in Xs]
    with pytest.raises(lib.AdagioError) as e:
        ctx.fit_batched(dX, epss)
    assert e.value.code == lib.E_NONFINITE
    with pytest.raises(lib.AdagioError) as e:
        ctx.fit_batched(dX[:1], [1.5])
    assert e.value.code == lib.E_INVALID_ARG
    # the context stays usable
    res = ctx.fit_batched([dX[0]], [0.3])
    assert res[0]["status"] in (0, lib.E_NOT_CERTIFIABLE)
    n = Xs[0].shape[0]
    assert res[0]["cert"].pairs == n * (n - 1) // 2


@pytest.mark.slow
def test_batched_workload_64_instances(ctx):
    """The 64-instance ragged workload (n in [500, 20000], d in {128..1024})."""
    wls = synth.batched()
    dX = [torch.from_numpy(w.X).cuda() for w in wls]
    epss = [w.eps for w in wls]
    res = ctx.fit_batched(dX, epss, precision=1, graph=True)
    certified = 0
    for w, r in zip(wls, res):
        # flat spectra (small alpha) may not reach eps even at m = d
        if r["status"] == 0:
            assert r["cert"].max <= w.eps
            certified += 1
        else:
            assert r["status"] == -7 and r["m"] == w.X.shape[1] and r["cert"].max > w.eps
        assert r["cert"].pairs == w.X.shape[0] * (w.X.shape[0] - 1) // 2
    assert certified >= 32
    # every instance's certificate against the oracle's certificate of the
    # same (X, Y), all pairs (about 1.7e9 over the batch)
    for w, r in zip(wls, res):
        Y = ctx.embed(r["A"], torch.from_numpy(w.X).cuda()).cpu().numpy()
        o = certificate(w.X, Y, w.eps)
        assert_cert_parity(r["cert"], o, w.X, Y)
    # a sample of instances against the single fit
    for i in (0, 17, 40, 63):
        A, m, s, c, rc = ctx.fit(dX[i], eps=epss[i], precision=1)
        assert (res[i]["m"], res[i]["s"], res[i]["status"]) == (m, s, rc)
        assert torch.equal(res[i]["A"], A)
        _same_cert(res[i]["cert"], c)


def test_batched_features_match_single_call(ctx):
    """The predictor's features taken from each batched fit's own PCA agree with
    adagio_features on the same data (same spectrum up to the iteration's
    tolerance; log n, log d, eps and the constant exactly)."""
    rng = np.random.default_rng(23)
    Xs, epss = [], []
    for n in (900, 2500, 400):
        X, eps = synth.mnist_like_family(rng, n, d=196)
        Xs.append(X)
        epss.append(eps)
    dX = [torch.from_numpy(X).cuda() for X in Xs]
    res = ctx.fit_batched(dX, epss, features=True)
    for X, eps, r in zip(Xs, epss, res):
        f = ctx.features(X, eps)
        np.testing.assert_allclose(r["feats"][:16], f[:16], atol=2e-3)
        np.testing.assert_array_equal(r["feats"][64:], f[64:])
