"""Parity of the GPU k-nearest-neighbour search (Sec. 4.6, Sec. 4.7) with the FP64 oracle.

The oracle computes every distance from coordinate differences in FP64 and
orders by (distance, index); the GPU must return the same index lists, bit for
bit, and squared distances within FP64 rounding.
"""
import numpy as np
import pytest

from oracle import adagio as O
from oracle.knn import knn as oracle_knn
from paper_1609_05388_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1609_05388_gb300 import adagio as lib
    c = lib.Context(0)
    yield c
    c.close()


def check(idx, d2, ref_idx, ref_d2):
    idx = idx.cpu().numpy() if hasattr(idx, "cpu") else idx
    d2 = d2.cpu().numpy() if hasattr(d2, "cpu") else d2
    np.testing.assert_array_equal(idx, ref_idx)
    np.testing.assert_allclose(d2, ref_d2, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("n,m,k", [(1500, 20, 10), (1031, 1, 1), (2000, 64, 30), (700, 37, 48)])
def test_graph_of_one_point_set(ctx, n, m, k):
    rng = np.random.default_rng(n + m)
    Y = rng.standard_normal((n, m)).astype(np.float32)
    idx, d2 = ctx.knn(torch.from_numpy(Y).cuda(), k)
    ref_idx, ref_d2 = oracle_knn(Y, Y, k, exclude_self=True)
    check(idx, d2, ref_idx, ref_d2)


def test_queries_against_a_separate_base(ctx):
    rng = np.random.default_rng(7)
    B = rng.standard_normal((2000, 64)).astype(np.float32) * np.linspace(3.0, 0.1, 64).astype(np.float32)
    Q = rng.standard_normal((300, 64)).astype(np.float32)
    idx, d2 = ctx.knn(Q, 30, B=B)                      # host arrays
    ref_idx, ref_d2 = oracle_knn(Q, B, 30)
    check(idx, d2, ref_idx, ref_d2)


def test_duplicates_and_ties_by_index(ctx):
    rng = np.random.default_rng(8)
    base = rng.integers(-3, 4, size=(400, 5)).astype(np.float32)  # many equal distances
    Y = np.concatenate([base, base[:50]], axis=0)                  # exact duplicates
    idx, d2 = ctx.knn(torch.from_numpy(Y).cuda(), 12)
    ref_idx, ref_d2 = oracle_knn(Y, Y, 12, exclude_self=True)
    check(idx, d2, ref_idx, ref_d2)


def test_on_a_certified_embedding(ctx):
    """The workload of the applications: neighbours in the embedded space of
    an MNIST-shaped set under the map the library fits."""
    wl = synth.mnist_like(seed=1, n=5000)
    f = O.fit(wl.X.astype(np.float64), 150, 3)
    Y = O.embed(f.A, wl.X).astype(np.float32)
    idx, d2 = ctx.knn(torch.from_numpy(Y).cuda(), 30)
    ref_idx, ref_d2 = oracle_knn(Y, Y, 30, exclude_self=True)
    check(idx, d2, ref_idx, ref_d2)


def test_full_size_graph_sampled(ctx):
    """60 000 x 421 (the benchmark's embedding dimension), k = 30: the full
    graph on the GPU, 256 sampled rows by the oracle."""
    wl = synth.mnist_like(seed=1)
    rng = np.random.default_rng(0)
    A = (rng.standard_normal((421, 784)) / np.sqrt(421)).astype(np.float32)
    Xd = torch.from_numpy(wl.X).cuda()
    Y = ctx.embed(A, Xd)
    idx, d2 = ctx.knn(Y, 30)
    Yh = Y.cpu().numpy()
    rows = rng.choice(Yh.shape[0], 256, replace=False)
    ref_idx, ref_d2 = oracle_knn(Yh[rows], Yh, 31)
    for r, q in enumerate(rows):
        keep = ref_idx[r] != q
        ri, rd = ref_idx[r][keep][:30], ref_d2[r][keep][:30]
        np.testing.assert_array_equal(idx[q].cpu().numpy(), ri)
        np.testing.assert_allclose(d2[q].cpu().numpy(), rd, rtol=1e-12)
    assert ctx.knn_last_exact_rows() <= Yh.shape[0] // 100


def test_bad_arguments(ctx):
    from paper_1609_05388_gb300 import adagio as lib
    Y = np.ones((10, 3), dtype=np.float32)
    for k in (0, 49, 10):
        with pytest.raises(lib.AdagioError) as ei:
            ctx.knn(Y, k)
        assert ei.value.code == lib.E_INVALID_ARG
    idx, _ = ctx.knn(np.arange(10, dtype=np.float32).reshape(10, 1), 9)
    assert idx.shape == (10, 9)
    Z = np.ones((40, 3), dtype=np.float32)
    Z[7, 1] = np.nan
    with pytest.raises(lib.AdagioError) as ei:
        ctx.knn(Z, 3)
    assert ei.value.code == lib.E_NONFINITE
