"""The allocation-free certificate matches adagio_distortion (collected last).

adagio_distortion_noalloc serves callers that cannot let the library allocate
device memory during a call (a service whose device memory belongs to its own
pool, a loop that cannot take cudaMalloc's device-wide synchronisation).  It
computes the FP32 certificate inside a fixed static scratch array.  This test
calls it through the C ABI twice in a row on different data -- the second call
must not see the first call's leftovers in the shared scratch -- and compares
each result with adagio_distortion's and with the FP64 oracle, within the
tolerances every other certificate test uses.
"""
import numpy as np
import pytest

from gpu_helpers import assert_cert_parity
from oracle.certificate import certificate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(seed, n, d, m):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((n, d)) * np.linspace(3.0, 0.2, d)[None, :]).astype(np.float32)
    X[5] = X[2]                                   # one degenerate pair
    A = rng.standard_normal((m, d)) / np.sqrt(m)
    Y = (X.astype(np.float64) @ A.T).astype(np.float32)
    return X, Y


def test_noalloc_matches_distortion_on_two_calls_in_a_row():
    from paper_1609_05388_gb300 import adagio as lib
    with lib.Context(0) as ctx:
        for seed, (n, d, m, eps) in enumerate([(1000, 300, 120, 0.3), (777, 64, 16, 0.5)]):
            X, Y = _case(seed, n, d, m)
            Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
            a = ctx.distortion_noalloc(Xd, Yd, eps)
            b = ctx.distortion(Xd, Yd, eps, precision=lib.PREC_FP32)
            o = certificate(X, Y, eps)
            assert_cert_parity(a, o, X, Y)
            assert a.pairs == b.pairs and a.degenerate == b.degenerate == 1
            assert abs(a.max - b.max) <= 1e-5 and abs(a.mean - b.mean) <= 1e-6
            assert int(np.abs(a.hist - b.hist).sum()) <= 2 * o.near_edge
            assert abs(a.violations - b.violations) <= o.near_edge


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_1609_05388_gb300 import adagio as lib
    with lib.Context(0) as ctx:
        X = torch.zeros((1025, 8), device="cuda")
        with pytest.raises(lib.AdagioError) as ei:
            ctx.distortion_noalloc(X, X, 0.1)
        assert ei.value.code == lib.E_INVALID_ARG
        X = torch.zeros((100, 513), device="cuda")
        Y = torch.zeros((100, 8), device="cuda")
        with pytest.raises(lib.AdagioError) as ei:
            ctx.distortion_noalloc(X, Y, 0.1)
        assert ei.value.code == lib.E_INVALID_ARG
