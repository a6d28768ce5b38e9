"""Pins for the oracle's all-pairs certificate (Eq. 2 and Eq. 3) -- CPU only.

Each pin is fixed by something other than the oracle itself: a worked example
whose distances are computed by hand, closed-form distortions of scalings and
isometries, invariances of Eq. 2, and the pair-count identity.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle.certificate import certificate, pair_distortion

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _three_point():
    xs, ys, pairs, mx = [], [], [], None
    with open(os.path.join(GOLDEN, "three_point.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            t = line.split()
            if t[0] == "x":
                xs.append([float(v) for v in t[1:]])
            elif t[0] == "y":
                ys.append([float(v) for v in t[1:]])
            elif t[0] == "pair":
                pairs.append((int(t[1]), int(t[2]), t[3]))
            elif t[0] == "max":
                mx = (float(t[1]), int(t[2]), int(t[3]))
    return np.array(xs), np.array(ys), pairs, mx


def _closed(expr):
    return {"0": 0.0, "0.5": 0.5, "1-sqrt(13)/5": 1.0 - math.sqrt(13.0) / 5.0}[expr]


def test_three_point_worked_example():
    X, Y, pairs, (mx, ai, aj) = _three_point()
    c = certificate(X, Y, eps=0.3, lo=0.0, hi=1.0, nbins=4, threads=2)
    assert c.pairs == 3 and c.degenerate == 0
    assert c.max == pytest.approx(mx, abs=1e-15)
    assert (c.argmax_i, c.argmax_j) == (ai, aj)
    vals = [_closed(e) for _, _, e in pairs]
    assert c.mean == pytest.approx(sum(vals) / 3, abs=1e-15)
    # bins of width 1/4: 0 -> bin 0, 0.2789 -> bin 1, 0.5 -> bin 2
    assert list(c.hist) == [1, 1, 1, 0]
    assert c.violations == 1          # only 0.5 > 0.3
    got = pair_distortion(X, Y, [p[0] for p in pairs], [p[1] for p in pairs])
    np.testing.assert_allclose(got, vals, atol=1e-15)


@pytest.mark.parametrize("scale", [0.75, 1.25, 2.0])
def test_uniform_scaling_has_closed_form_distortion(scale):
    rng = np.random.default_rng(3)
    X = rng.integers(-8, 8, size=(40, 5)).astype(np.float64)
    X = np.unique(X, axis=0)
    n = X.shape[0]
    c = certificate(X, scale * X, eps=abs(scale - 1.0), lo=0.0, hi=2.0, nbins=64)
    assert c.pairs == n * (n - 1) // 2
    assert c.max == pytest.approx(abs(scale - 1.0), abs=1e-15)
    assert c.mean == pytest.approx(abs(scale - 1.0), abs=1e-14)
    # distortion exactly eps is not a violation (strict >)
    assert c.violations == 0
    c2 = certificate(X, scale * X, eps=abs(scale - 1.0) - 1e-9, lo=0.0, hi=2.0)
    assert c2.violations == c.pairs


def test_isometry_has_zero_distortion():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((60, 7))
    Q, _ = np.linalg.qr(rng.standard_normal((7, 7)))
    c = certificate(X, X @ Q + 5.0, eps=1e-6, lo=0.0, hi=1e-3, nbins=8)
    assert c.max < 1e-12
    assert c.violations == 0
    assert c.hist[0] == c.pairs


def test_translation_and_scale_invariance():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((70, 6))
    Y = X @ rng.standard_normal((6, 3))
    a = certificate(X, Y, eps=0.5, lo=0.0, hi=2.0)
    b = certificate(3.0 * X + 11.0, 3.0 * Y - 7.0, eps=0.5, lo=0.0, hi=2.0)
    assert b.max == pytest.approx(a.max, rel=1e-12)
    assert (b.argmax_i, b.argmax_j) == (a.argmax_i, a.argmax_j)
    assert b.mean == pytest.approx(a.mean, rel=1e-12)
    assert b.violations == a.violations


def test_duplicates_are_degenerate_and_counts_conserve():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((30, 4))
    X[7] = X[3]
    X[20] = X[3]
    X[11] = X[12]
    Y = X @ rng.standard_normal((4, 2))
    c = certificate(X, Y, eps=0.3, lo=0.0, hi=0.6)
    n = X.shape[0]
    assert c.pairs == n * (n - 1) // 2
    assert c.degenerate == 4        # {3,7,20} gives 3 pairs, {11,12} one
    assert int(c.hist.sum()) + c.overflow + c.degenerate == c.pairs


def test_row_ranges_partition_the_pairs():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((50, 5))
    Y = X @ rng.standard_normal((5, 3))
    full = certificate(X, Y, eps=0.4)
    parts = [certificate(X, Y, eps=0.4, rows=r) for r in [(0, 13), (13, 31), (31, 50)]]
    assert sum(p.pairs for p in parts) == full.pairs
    assert sum(p.violations for p in parts) == full.violations
    np.testing.assert_array_equal(sum(p.hist for p in parts), full.hist)
    assert max(p.max for p in parts) == full.max


def test_brute_force_tiny():
    """Cross-check against an independent double loop on a tiny input."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((25, 4))
    Y = X @ rng.standard_normal((4, 2))
    deltas = {}
    for i, j in itertools.combinations(range(25), 2):
        dx = math.dist(X[i], X[j])
        dy = math.dist(Y[i], Y[j])
        deltas[(i, j)] = abs(dy / dx - 1.0)
    c = certificate(X, Y, eps=0.5, lo=0.0, hi=1.0, nbins=10)
    assert c.max == pytest.approx(max(deltas.values()), rel=1e-12)
    assert c.violations == sum(v > 0.5 for v in deltas.values())
    ref = np.zeros(10, dtype=np.int64)
    over = 0
    for v in deltas.values():
        if v >= 1.0:
            over += 1
        else:
            ref[int(v * 10)] += 1
    np.testing.assert_array_equal(c.hist, ref)
    assert c.overflow == over


@pytest.mark.parametrize("offset,near", [(-2e-6, 0), (-5e-7, 1), (5e-7, 1), (2e-6, 0)])
@pytest.mark.parametrize("target", ["edge", "eps"])
def test_near_edge_counts_pairs_within_1e6_of_an_edge_or_eps(offset, near, target):
    """One pair with a hand-placed distortion: 1-D points 0 and 1 mapped to 0
    and 1 + delta have distortion exactly delta (up to FP64 rounding, ~1e-16).
    near_edge counts it when delta lies within 1e-6 of a bin edge or of eps,
    and the histogram puts it on the correct side of the edge."""
    lo, hi, nbins = 0.0, 0.5, 64
    w = (hi - lo) / nbins                     # 0.0078125: edges at multiples of w
    if target == "edge":
        eps = 0.2                              # 0.2 / w = 25.6: eps is not an edge
        base = 20 * w                          # the lower edge of bin 20
    else:
        eps = 0.2
        base = eps
    delta = base + offset
    X = np.array([[0.0], [1.0]])
    Y = np.array([[0.0], [1.0 + delta]])
    c = certificate(X, Y, eps=eps, lo=lo, hi=hi, nbins=nbins)
    assert c.pairs == 1 and c.degenerate == 0
    assert c.max == pytest.approx(delta, abs=1e-15)
    assert c.near_edge == near
    assert int(np.argmax(c.hist)) == int(math.floor(delta / w)) and c.hist.sum() == 1
    if target == "edge":
        assert int(np.argmax(c.hist)) == (20 if offset > 0 else 19)
    assert c.violations == (1 if delta > eps else 0)


def test_tile_ranges_partition_the_pairs_and_match_row_ranges():
    """Tile ranges of the row-major tile triangle partition the pairs: any cut
    of [0, T(T+1)/2) into ranges gives parts that add up to the whole
    certificate, and the tiles of whole block rows are exactly a row range."""
    rng = np.random.default_rng(9)
    n, tile = 53, 8                               # 7 block rows, a ragged last block
    X = rng.standard_normal((n, 4))
    Y = X @ rng.standard_normal((4, 3))
    from oracle.certificate import certificate_tiles
    full = certificate(X, Y, eps=0.4)
    T = (n + tile - 1) // tile
    ntp = T * (T + 1) // 2
    cuts = [0, 3, 4, 11, 19, ntp]
    parts = [certificate_tiles(X, Y, 0.4, a, b, tile=tile) for a, b in zip(cuts[:-1], cuts[1:])]
    assert sum(p.pairs for p in parts) == full.pairs == n * (n - 1) // 2
    assert sum(p.violations for p in parts) == full.violations
    np.testing.assert_array_equal(sum(p.hist for p in parts), full.hist)
    assert max(p.max for p in parts) == full.max
    # block rows 0..1 are tiles [0, T + T - 1): rows [0, 2 tile)
    a = certificate_tiles(X, Y, 0.4, 0, T + (T - 1), tile=tile)
    b = certificate(X, Y, eps=0.4, rows=(0, 2 * tile))
    assert (a.pairs, a.violations, a.max) == (b.pairs, b.violations, b.max)
    np.testing.assert_array_equal(a.hist, b.hist)
    # a single tile (I, J) = (1, 3): 8 x 8 pairs
    t13 = T + (3 - 1)
    one = certificate_tiles(X, Y, 0.4, t13, t13 + 1, tile=tile)
    assert one.pairs == tile * tile
    # more block rows than the points need (blocks past n hold no pairs)
    T2 = T + 1
    whole = certificate_tiles(X, Y, 0.4, 0, T2 * (T2 + 1) // 2, tile=tile, blocks=T2)
    assert whole.pairs == full.pairs and whole.max == full.max
