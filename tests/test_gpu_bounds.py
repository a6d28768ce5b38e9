"""The certificate's per-pair error bound holds (and how tight it is), per arithmetic.

For the first tile pairs the tile kernel visits, the library reports its fast
squared distances dx2, dy2 and their bounds ex, ey.  Every valid pair must
satisfy |dx2 - exact| <= ex and |dy2 - exact| <= ey, with the exact squared
distances from the float32 inputs in float64.  A pair whose bound fails could
be binned wrongly without being recomputed, so this is the soundness check of
the fast path.
"""
import numpy as np
import pytest

from oracle import adagio as O
from paper_1609_05388_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1609_05388_gb300 import adagio as lib
    c = lib.Context(0)
    yield c
    c.close()


def exact_sqdist_block(Z, rows, cols):
    Z = Z.astype(np.float64)
    Zc = Z - Z.mean(axis=0)
    a, b = Zc[rows], Zc[cols]
    return (np.sum(a * a, 1)[:, None] + np.sum(b * b, 1)[None, :] - 2.0 * a @ b.T)


def workload(name):
    if name == "mnist":
        X = synth.mnist_like(seed=1, n=1500).X
        m = 150
    elif name == "small":
        X = synth.small(seed=0, n=1500).X
        m = 20
    else:
        X = synth.power_law(np.random.default_rng(2), 1500, 512, 1.0)
        m = 96
    f = O.fit(X.astype(np.float64), m, 3)
    Y = O.embed(f.A, X).astype(np.float32)
    return X, Y


@pytest.mark.parametrize("prec,kernel", [(0, 0), (1, 1), (1, 2), (2, 1), (2, 2)])
@pytest.mark.parametrize("name", ["mnist", "small", "powerlaw"])
def test_fast_path_error_bound(ctx, prec, kernel, name):
    ctx.set_tile_kernel(kernel)
    X, Y = workload(name)
    n = X.shape[0]
    T = (n + 127) // 128
    tiles = min(T * (T + 1) // 2, 30)
    out, ij = ctx.debug_tile_bounds(X, Y, tiles, precision=prec)
    worst_x = worst_y = 0.0
    rx, ry = [], []
    for t in range(tiles):
        I, J = int(ij[t, 0]), int(ij[t, 1])
        rows = I * 128 + np.arange(128)
        cols = J * 128 + np.arange(128)
        valid = (rows[:, None] < cols[None, :]) & (cols[None, :] < n)
        r_ok, c_ok = np.minimum(rows, n - 1), np.minimum(cols, n - 1)
        ex_x = exact_sqdist_block(X, r_ok, c_ok)
        ex_y = exact_sqdist_block(Y, r_ok, c_ok)
        blk = out[t]
        ratio_x = np.abs(blk[..., 0] - ex_x) / blk[..., 2]
        ratio_y = np.abs(blk[..., 1] - ex_y) / blk[..., 3]
        rx.append(ratio_x[valid])
        ry.append(ratio_y[valid])
    rx, ry = np.concatenate(rx), np.concatenate(ry)
    print(f"\n[bound] prec={prec} kernel={kernel} {name}: |err|/bound x max {rx.max():.3f} p99.9 "
          f"{np.quantile(rx, 0.999):.3f} median {np.median(rx):.4f}; "
          f"y max {ry.max():.3f} p99.9 {np.quantile(ry, 0.999):.3f} median {np.median(ry):.4f}")
    assert rx.max() <= 1.0 and ry.max() <= 1.0
