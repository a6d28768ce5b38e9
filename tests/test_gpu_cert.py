"""Parity of the GPU all-pairs certificate (Eq. 2, Eq. 3) with the FP64 oracle."""
import numpy as np
import pytest

from gpu_helpers import CERT_MODES, assert_cert_parity
from oracle import adagio as O
from oracle.certificate import certificate, certificate_tiles, pair_distortion
from paper_1609_05388_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1609_05388_gb300 import adagio as lib
    c = lib.Context(0)
    yield c
    c.close()


def oracle_embedding(X, m, seed=3):
    f = O.fit(X.astype(np.float64), m, seed)
    return O.embed(f.A, X).astype(np.float32)


def run(ctx, X, Y, eps, prec, lo=0.0, hi=0.0, device=True, tiles=0):
    ctx.set_tile_kernel(tiles)
    if device:
        Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
        return ctx.distortion(Xd, Yd, eps, lo, hi, precision=prec)
    return ctx.distortion(X, Y, eps, lo, hi, precision=prec)


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
def test_small_workload(ctx, prec, tiles):
    wl = synth.small(seed=0)                     # 2000 x 64, 1 999 000 pairs
    Y = oracle_embedding(wl.X, 20)
    g = run(ctx, wl.X, Y, 0.2, prec, tiles=tiles)
    o = certificate(wl.X, Y, 0.2)
    assert_cert_parity(g, o, wl.X, Y)


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
def test_mnist_shaped_ragged(ctx, prec, tiles):
    wl = synth.mnist_like(seed=1, n=3000)        # 23 full tiles + a ragged one
    Y = oracle_embedding(wl.X, 150)
    g = run(ctx, wl.X, Y, 0.1, prec, tiles=tiles)
    o = certificate(wl.X, Y, 0.1)
    assert_cert_parity(g, o, wl.X, Y)


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
@pytest.mark.parametrize("n", [2, 3, 127, 128, 129, 300])
def test_tiny_and_tile_edges(ctx, prec, tiles, n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, 37)).astype(np.float32)
    Y = (X @ rng.standard_normal((37, 11)) / np.sqrt(11)).astype(np.float32)
    g = run(ctx, X, Y, 0.3, prec, 0.0, 2.0, tiles=tiles)
    o = certificate(X, Y, 0.3, 0.0, 2.0)
    assert_cert_parity(g, o, X, Y)


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
def test_host_and_device_pointers_agree(ctx, prec, tiles):
    wl = synth.small(seed=0, n=900)
    Y = oracle_embedding(wl.X, 12)
    a = run(ctx, wl.X, Y, 0.2, prec, device=True, tiles=tiles)
    b = run(ctx, wl.X, Y, 0.2, prec, device=False, tiles=tiles)
    assert a.max == b.max and np.array_equal(a.hist, b.hist) and a.violations == b.violations


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
def test_duplicates_are_degenerate(ctx, prec, tiles):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((400, 16)).astype(np.float32)
    X[10] = X[3]
    X[200] = X[3]
    X[399] = X[0]
    Y = (X @ rng.standard_normal((16, 8)) / np.sqrt(8)).astype(np.float32)
    g = run(ctx, X, Y, 0.5, prec, 0.0, 4.0, tiles=tiles)
    o = certificate(X, Y, 0.5, 0.0, 4.0)
    assert o.degenerate == 4
    assert_cert_parity(g, o, X, Y)


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
def test_all_points_identical(ctx, prec, tiles):
    X = np.full((50, 5), 0.25, dtype=np.float32)
    Y = np.zeros((50, 2), dtype=np.float32)
    g = run(ctx, X, Y, 0.1, prec, tiles=tiles)
    assert g.degenerate == g.pairs == 50 * 49 // 2
    assert g.max == 0.0 and int(g.hist.sum()) == 0


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
def test_one_dimensional(ctx, prec, tiles):
    rng = np.random.default_rng(6)
    X = rng.standard_normal((257, 1)).astype(np.float32)
    Y = (1.5 * X).astype(np.float32)
    g = run(ctx, X, Y, 0.6, prec, 0.0, 1.0, tiles=tiles)
    o = certificate(X, Y, 0.6, 0.0, 1.0)
    assert_cert_parity(g, o, X, Y)


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
def test_pairs_exactly_on_an_edge(ctx, prec, tiles):
    # Y = 1.25 X: every pair has distortion exactly 0.25 = eps = edge of bin 32
    rng = np.random.default_rng(7)
    X = rng.integers(-50, 50, size=(300, 6)).astype(np.float32)
    X = np.unique(X, axis=0)
    Y = (1.25 * X).astype(np.float32)
    g = run(ctx, X, Y, 0.25, prec, tiles=tiles)
    o = certificate(X, Y, 0.25)
    assert o.near_edge == o.pairs
    assert_cert_parity(g, o, X, Y)


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
def test_pairs_just_off_a_large_edge(ctx, prec, tiles):
    # Y ~ 1.7500012 X: distortions scatter within a few 1e-7 of 0.7500012, just
    # above eps = 0.75 (the edge of bin 32).  At this distortion the
    # recompute's first level bounds its error by ~1.3e-6, more than the 1e-6
    # band, so pairs between 1e-6 and that bound from the edge are settled by
    # its exact second level; every pair farther than 1e-6 must count exactly.
    rng = np.random.default_rng(17)
    X = np.unique(rng.integers(-8, 9, size=(300, 6)).astype(np.float32), axis=0)
    Y = (np.float32(1.7500012) * X).astype(np.float32)
    g = run(ctx, X, Y, 0.75, prec, tiles=tiles)
    o = certificate(X, Y, 0.75)
    assert o.near_edge < o.pairs
    assert_cert_parity(g, o, X, Y)


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
def test_nonfinite_input_rejected(ctx, prec, tiles):
    from paper_1609_05388_gb300 import adagio as lib
    X = np.ones((10, 3), dtype=np.float32)
    X[4, 1] = np.nan
    Y = np.ones((10, 2), dtype=np.float32)
    with pytest.raises(lib.AdagioError) as ei:
        run(ctx, X, Y, 0.1, prec, tiles=tiles)
    assert ei.value.code == lib.E_NONFINITE


def test_bad_arguments_rejected(ctx):
    from paper_1609_05388_gb300 import adagio as lib
    X = np.ones((10, 3), dtype=np.float32)
    for eps in (0.0, 1.0, -0.5, float("nan")):
        with pytest.raises(lib.AdagioError) as ei:
            ctx.distortion(X, X, eps)
        assert ei.value.code == lib.E_INVALID_ARG
    with pytest.raises(lib.AdagioError):
        ctx.distortion(X[:1], X[:1], 0.1)
    with pytest.raises(lib.AdagioError):
        ctx.distortion(X, X, 0.1, precision=7)


@pytest.mark.parametrize("prec,tiles", CERT_MODES)
def test_full_size_mnist_shaped_sampled(ctx, prec, tiles):
    """60 000 x 784 (1.8e9 pairs): properties at full size, sampled pairs by the oracle."""
    wl = synth.mnist_like(seed=1)
    m = 200
    rng = np.random.default_rng(0)
    # the embedding comes from the oracle's map of a 4000-point sample
    f = O.fit(wl.X[:4000].astype(np.float64), m, 3)
    Y = (wl.X.astype(np.float64) @ f.A.T).astype(np.float32)
    g = run(ctx, wl.X, Y, 0.1, prec, tiles=tiles)
    assert g.pairs == 60000 * 59999 // 2
    assert int(g.hist.sum()) + g.overflow + g.degenerate == g.pairs
    d_arg = pair_distortion(wl.X, Y, [g.argmax_i], [g.argmax_j])[0]
    assert abs(d_arg - g.max) <= 1e-5
    I = rng.integers(0, 60000, 400000)
    J = rng.integers(0, 60000, 400000)
    keep = I != J
    dl = pair_distortion(wl.X, Y, I[keep], J[keep])
    dl = dl[np.isfinite(dl)]
    assert dl.max() <= g.max + 1e-5
    # sampled violation and bin fractions agree with the exhaustive counts (6 sigma)
    good = g.pairs - g.degenerate
    p_hat = np.mean(dl > 0.1)
    p = g.violations / good
    assert abs(p - p_hat) <= 6 * np.sqrt(max(p * (1 - p), 1e-12) / dl.size) + 1e-6
    assert abs(g.mean - dl.mean()) <= 6 * dl.std() / np.sqrt(dl.size)


def test_tile_kernels_agree(ctx):
    """Single-CTA and CTA-pair tiles, in any schedule band, classify every pair the same way."""
    from paper_1609_05388_gb300 import adagio as lib
    wl = synth.mnist_like(seed=1, n=5000)
    Y = oracle_embedding(wl.X, 150)
    o = certificate(wl.X, Y, 0.1)
    res = []
    for tiles, band in ((lib.TILES_SINGLE, 0), (lib.TILES_PAIR, 0), (lib.TILES_SINGLE, 4),
                        (lib.TILES_SINGLE, 16), (lib.TILES_PAIR, 16)):
        ctx.set_tile_kernel(tiles, band)
        res.append(ctx.distortion(torch.from_numpy(wl.X).cuda(), torch.from_numpy(Y).cuda(), 0.1,
                                  precision=lib.PREC_FP16X3))
        assert_cert_parity(res[-1], o, wl.X, Y)
    a = res[0]
    for b in res[1:]:
        assert a.max == b.max and (a.argmax_i, a.argmax_j) == (b.argmax_i, b.argmax_j)
        assert int(np.abs(a.hist - b.hist).sum()) <= 2 * o.near_edge
        assert abs(a.mean - b.mean) <= 1e-9
    ctx.set_tile_kernel(lib.TILES_AUTO)
    assert ctx.tile_kernel_for(60000) in (lib.TILES_SINGLE, lib.TILES_PAIR)
    assert ctx.tile_kernel_for(1000) == lib.TILES_SINGLE


def test_strided_host_inputs_match_contiguous(ctx):
    """Host arrays with a row stride larger than their width (the C ABI's ldx,
    ldy) are staged by a pitched copy; contiguous ones by a linear copy.  Both
    give the same certificate, bit for bit."""
    import ctypes
    from paper_1609_05388_gb300 import adagio as lib
    rng = np.random.default_rng(23)
    n, d, m = 700, 37, 13
    X = rng.standard_normal((n, d)).astype(np.float32)
    Y = (X @ rng.standard_normal((d, m)).astype(np.float32) / np.sqrt(m)).astype(np.float32)
    Xw = np.zeros((n, d + 5), dtype=np.float32)
    Yw = np.zeros((n, m + 3), dtype=np.float32)
    Xw[:, :d] = X
    Yw[:, :m] = Y
    ref = ctx.distortion(X, Y, 0.3, precision=1)
    c = lib.CertStruct()
    rc = lib.LIB.adagio_distortion(ctx.h, Xw.ctypes.data, n, d, d + 5, Yw.ctypes.data, m, m + 3,
                                   0.3, 0.0, 0.0, 1, ctypes.byref(c), None)
    assert rc == 0
    got = lib.Certificate.from_struct(c)
    assert got.max == ref.max and got.mean == ref.mean
    assert np.array_equal(got.hist, ref.hist) and got.violations == ref.violations


def test_unaligned_device_rows_match_contiguous(ctx):
    """Device views whose row stride is not a multiple of 4 floats are
    re-pitched to 16-byte aligned rows before the certificate; the result is
    the one of the contiguous arrays, bit for bit."""
    import torch
    rng = np.random.default_rng(29)
    n, d, m = 650, 21, 11
    X = rng.standard_normal((n, d)).astype(np.float32)
    Y = (X @ rng.standard_normal((d, m)).astype(np.float32) / np.sqrt(m)).astype(np.float32)
    Xw = torch.zeros((n, d + 2), dtype=torch.float32, device="cuda")
    Yw = torch.zeros((n, m + 1), dtype=torch.float32, device="cuda")
    Xw[:, :d] = torch.from_numpy(X).cuda()
    Yw[:, :m] = torch.from_numpy(Y).cuda()
    ref = ctx.distortion(X, Y, 0.3, precision=1)
    got = ctx.distortion(Xw[:, :d], Yw[:, :m], 0.3, precision=1)
    torch.cuda.synchronize()
    assert got.max == ref.max and got.mean == ref.mean
    assert np.array_equal(got.hist, ref.hist) and got.violations == ref.violations


@pytest.mark.parametrize("prec", [1, 2])
def test_full_size_large_sampled(ctx, prec):
    """200 000 x 2048 (2.0e10 pairs, the largest synthetic workload: power-law
    spectrum plus Laplace outliers): properties at full size, sampled pairs by
    the oracle.  The map is a JL matrix of m = 300 rows, the oracle's bit for bit."""
    wl = synth.large(seed=4)
    n, d, m = wl.X.shape[0], wl.X.shape[1], 300
    S = ctx.jl_matrix(9, m, d)
    assert np.array_equal(S, O.jl_matrix(9, m, d).astype(np.float32))
    Xd = torch.from_numpy(wl.X).cuda()
    Y = (Xd @ torch.from_numpy(S).cuda().T).contiguous()
    g = ctx.distortion(Xd, Y, 0.1, precision=prec)
    Yh = Y.cpu().numpy()
    assert g.pairs == n * (n - 1) // 2
    assert int(g.hist.sum()) + g.overflow + g.degenerate == g.pairs
    d_arg = pair_distortion(wl.X, Yh, [g.argmax_i], [g.argmax_j])[0]
    assert abs(d_arg - g.max) <= 1e-5
    rng = np.random.default_rng(5)
    I = rng.integers(0, n, 100000)
    J = rng.integers(0, n, 100000)
    keep = I != J
    dl = pair_distortion(wl.X, Yh, I[keep], J[keep])
    dl = dl[np.isfinite(dl)]
    assert dl.max() <= g.max + 1e-5
    good = g.pairs - g.degenerate
    p_hat = np.mean(dl > 0.1)
    p = g.violations / good
    assert abs(p - p_hat) <= 6 * np.sqrt(max(p * (1 - p), 1e-12) / dl.size) + 1e-6
    assert abs(g.mean - dl.mean()) <= 6 * dl.std() / np.sqrt(dl.size)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_sharded_certificate_matches_whole(ctx, prec):
    """Shards of the tile triangle, certified one by one and merged, give the
    whole certificate: counts, histogram, recomputed pairs, maximum and its
    pair bit for bit, the mean to rounding."""
    from paper_1609_05388_gb300 import adagio as lib
    wl = synth.mnist_like(seed=1, n=3001)
    Y = oracle_embedding(wl.X, 120)
    X, Yd = torch.from_numpy(wl.X).cuda(), torch.from_numpy(Y).cuda()
    whole = ctx.distortion(X, Yd, 0.1, precision=prec)
    o = certificate(wl.X, Y, 0.1)
    assert_cert_parity(whole, o, wl.X, Y)
    for k in (2, 3, 7):
        parts = [ctx.distortion_shard(X, Yd, 0.1, s, k, precision=prec) for s in range(k)]
        assert sum(p.pairs for p in parts) == whole.pairs
        g = lib.cert_merge(parts)
        assert (g.pairs, g.degenerate, g.violations, g.overflow, g.recomputed) == \
            (whole.pairs, whole.degenerate, whole.violations, whole.overflow, whole.recomputed)
        assert np.array_equal(g.hist, whole.hist)
        assert (g.max, g.argmax_i, g.argmax_j) == (whole.max, whole.argmax_i, whole.argmax_j)
        assert abs(g.mean - whole.mean) <= 1e-12 * whole.mean
        assert_cert_parity(g, o, wl.X, Y)
        # every shard against the oracle's certificate of the same tiles
        n = wl.X.shape[0]
        B = 2 * (-(-n // 256))
        ntp = B * (B + 1) // 2
        for sh, part in enumerate(parts):
            t0, t1 = ntp * sh // k, ntp * (sh + 1) // k
            os_ = certificate_tiles(wl.X, Y, 0.1, t0, t1, blocks=B)
            assert (part.pairs, part.degenerate) == (os_.pairs, os_.degenerate)
            hist = np.array(part.hist[:], dtype=np.int64)
            assert int(np.abs(hist - os_.hist).sum()) <= 2 * os_.near_edge
            assert abs(part.violations - os_.violations) <= os_.near_edge
            assert abs(part.max - os_.max) <= 1e-5
            good = part.pairs - part.degenerate
            assert abs(part.sum / good - os_.mean) <= 1e-6
    with pytest.raises(lib.AdagioError):
        ctx.distortion_shard(X, Yd, 0.1, 3, 3, precision=prec)


def test_shards_of_two_points(ctx):
    """n = 2: three tiles, one pair; the shards without it are empty."""
    from paper_1609_05388_gb300 import adagio as lib
    X = np.array([[0.0, 0.0], [3.0, 4.0]], dtype=np.float32)
    Y = np.array([[0.0], [6.0]], dtype=np.float32)
    parts = [ctx.distortion_shard(X, Y, 0.5, s, 3, precision=1) for s in range(3)]
    assert [p.pairs for p in parts] == [1, 0, 0]
    g = lib.cert_merge(parts)
    assert g.pairs == 1 and abs(g.max - 0.2) <= 1e-6 and (g.argmax_i, g.argmax_j) == (0, 1)
