"""The allocation-free certificate matches adagio_distortion (collected last).

adagio_distortion_noalloc serves callers that cannot let the library allocate
device memory during a call (a service whose device memory belongs to its own
pool, a loop that cannot take cudaMalloc's device-wide synchronisation).  It
computes the FP32 certificate inside a fixed static scratch array.  These
tests call it through the C ABI twice in a row on different data -- the second
call must not see the first call's leftovers in the shared scratch -- and
compare each result with adagio_distortion's and with the FP64 oracle, within
the tolerances every other certificate test uses; they also run it at its
documented size limit, and check that it allocates nothing: the context's
workspace stays empty and the device's free memory does not change.
"""
import ctypes

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


def _noalloc_raw(lib, ctx, Xd, Yd, eps):
    """One call through the raw C symbol (no binding logic in between)."""
    c = lib.CertStruct()
    n, d = Xd.shape
    m = Yd.shape[1]
    rc = lib.LIB.adagio_distortion_noalloc(ctx.h, Xd.data_ptr(), n, d, d, Yd.data_ptr(), m, m,
                                           eps, 0.0, 0.0, ctypes.byref(c),
                                           torch.cuda.current_stream().cuda_stream)
    assert rc == 0, lib.LIB.adagio_last_error(ctx.h)
    return lib.Certificate.from_struct(c)


def test_noalloc_matches_distortion_on_two_calls_in_a_row():
    from paper_1609_05388_gb300 import adagio as lib
    with lib.Context(0) as ctx:
        for seed, (n, d, m, eps) in enumerate([(1000, 300, 120, 0.3), (777, 64, 16, 0.5)]):
            X, Y = _case(seed, n, d, m)
            Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
            a = _noalloc_raw(lib, ctx, Xd, Yd, eps)
            b = ctx.distortion(Xd, Yd, eps, precision=lib.PREC_FP32)
            o = certificate(X, Y, eps)
            assert_cert_parity(a, o, X, Y)
            assert a.pairs == b.pairs and a.degenerate == b.degenerate == 1
            assert abs(a.max - b.max) <= 1e-5 and abs(a.mean - b.mean) <= 1e-6
            assert int(np.abs(a.hist - b.hist).sum()) <= 2 * o.near_edge
            assert abs(a.violations - b.violations) <= o.near_edge


def test_noalloc_at_its_size_limit_allocates_nothing():
    """n = 1024, d = 512, m = 256 (the documented limit), two calls on fresh
    data after a set-up call: each matches the oracle; neither grows the
    context's workspace (it stays empty: nothing else ran on this context)
    nor changes the device's free memory."""
    from paper_1609_05388_gb300 import adagio as lib
    with lib.Context(0) as ctx:
        cases = [_case(10 + q, 1024, 512, 256) for q in range(3)]
        dev = [(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()) for X, Y in cases]
        torch.cuda.synchronize()
        _noalloc_raw(lib, ctx, *dev[0], 0.3)      # first call on the device: set-up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert ctx.workspace_bytes == 0
        for (X, Y), (Xd, Yd) in zip(cases[1:], dev[1:]):
            g = _noalloc_raw(lib, ctx, Xd, Yd, 0.3)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
            assert ctx.workspace_bytes == 0
            assert ctx.last_cert_stats()["grid"] > 0
            assert_cert_parity(g, certificate(X, Y, 0.3), X, Y)


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
        X = torch.zeros((100, 8), device="cuda")
        Y = torch.zeros((100, 257), device="cuda")
        with pytest.raises(lib.AdagioError) as ei:
            ctx.distortion_noalloc(X, Y, 0.1)
        assert ei.value.code == lib.E_INVALID_ARG
