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


def _full_size_ratios(ctx, X, Y, prec, frac):
    """|err| / bound of dx2 and dy2 over a strided `frac` of the 128 x 128 tiles
    of the full launch, against exact FP64 squared distances of the centred
    rows (coordinate differences, by the oracle)."""
    from oracle.certificate import pair_sqdist
    n = X.shape[0]
    B = 2 * (-(-n // 256))
    ntp = B * (B + 1) // 2
    stride = max(1, int(round(1.0 / frac)))
    tiles = (ntp - 1) // stride + 1
    rx, ry = [], []
    dev = torch.empty((tiles, 128, 128, 4), dtype=torch.float32, device="cuda")
    _, ij_all = ctx.debug_tile_bounds(X, Y, tiles, precision=prec, stride=stride, out=dev)
    torch.cuda.synchronize()
    for q0 in range(0, tiles, 256):
        cnt = min(256, tiles - q0)
        out = dev[q0:q0 + cnt].cpu().numpy()
        ij = ij_all[q0:q0 + cnt]
        I_all, J_all, sel = [], [], []
        for t in range(cnt):
            I, J = int(ij[t, 0]), int(ij[t, 1])
            rows = I * 128 + np.arange(128)
            cols = J * 128 + np.arange(128)
            valid = (rows[:, None] < cols[None, :]) & (cols[None, :] < n)
            a, b = np.nonzero(valid)
            I_all.append(rows[a]); J_all.append(cols[b]); sel.append((t, a, b))
        if not I_all:
            continue
        ex_x, ex_y = pair_sqdist(X, Y, np.concatenate(I_all), np.concatenate(J_all))
        off = 0
        for t, a, b in sel:
            blk = out[t]
            k = a.size
            rx.append(np.abs(blk[a, b, 0] - ex_x[off:off + k]) / blk[a, b, 2])
            ry.append(np.abs(blk[a, b, 1] - ex_y[off:off + k]) / blk[a, b, 3])
            off += k
    return np.concatenate(rx), np.concatenate(ry), tiles


@pytest.mark.slow
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_bound_at_full_size_mnist_shaped(ctx, prec):
    """1 % of the tiles of the 60 000 x 784 launch (about 1.2e7 pairs), the
    benchmark's map dimension m = 421."""
    wl = synth.mnist_like(seed=1)
    f = O.fit(wl.X[:4000].astype(np.float64), 421, 3)
    Y = (wl.X.astype(np.float64) @ f.A.T).astype(np.float32)
    ctx.set_tile_kernel(0)
    rx, ry, tiles = _full_size_ratios(ctx, wl.X, Y, prec, 0.01)
    print(f"\n[bound-full] mnist60k prec={prec} tiles={tiles} pairs={rx.size}: x max {rx.max():.3f} "
          f"p99.99 {np.quantile(rx, 0.9999):.3f}; y max {ry.max():.3f} p99.99 {np.quantile(ry, 0.9999):.3f}")
    # sound; the calibrated BF16x3 bound with a fourfold margin (FP32 and
    # FP16x3 carry worst-case bounds)
    lim = 1.0 if prec in (0, 1) else 0.25
    assert rx.max() <= lim and ry.max() <= lim


@pytest.mark.slow
@pytest.mark.parametrize("prec", [1, 2])
def test_bound_at_full_size_large(ctx, prec):
    """1 % of the tiles of the 200 000 x 2048 launch (about 2e8 pairs) under a
    JL map of 300 rows."""
    wl = synth.large(seed=4)
    n, d, m = wl.X.shape[0], wl.X.shape[1], 300
    S = ctx.jl_matrix(9, m, d)
    Xd = torch.from_numpy(wl.X).cuda()
    Y = (Xd @ torch.from_numpy(S).cuda().T).contiguous().cpu().numpy()
    del Xd
    ctx.set_tile_kernel(0)
    rx, ry, tiles = _full_size_ratios(ctx, wl.X, Y, prec, 0.01)
    print(f"\n[bound-full] large200k prec={prec} tiles={tiles} pairs={rx.size}: x max {rx.max():.3f} "
          f"p99.99 {np.quantile(rx, 0.9999):.3f}; y max {ry.max():.3f} p99.99 {np.quantile(ry, 0.9999):.3f}")
    # sound; the calibrated BF16x3 bound with a fourfold margin (FP32 and
    # FP16x3 carry worst-case bounds)
    lim = 1.0 if prec in (0, 1) else 0.25
    assert rx.max() <= lim and ry.max() <= lim
