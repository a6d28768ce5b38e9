"""Shared helpers of the GPU parity tests."""
import numpy as np
import pytest

from oracle.certificate import pair_distortion

# Arithmetic of the certificate tiles exercised by the parity tests.
PRECISIONS = (0, 1, 2)   # FP32 SIMT, FP16x3 and BF16x3 tensor cores

# (arithmetic, tile kernel) of the certificate parity tests: the FP32 SIMT
# tiles, and each split precision on single-CTA and CTA-pair tensor tiles
CERT_MODES = [pytest.param(0, 0, id="fp32"),
              pytest.param(1, 1, id="fp16x3-single"), pytest.param(1, 2, id="fp16x3-pair"),
              pytest.param(2, 1, id="bf16x3-single"), pytest.param(2, 2, id="bf16x3-pair")]


def assert_cert_parity(g, o, X, Y, max_tol=1e-5, mean_tol=1e-6):
    """GPU certificate g vs oracle certificate o of the same (X, Y).

    Bar: pair and degenerate counts exact; histogram, overflow and violation
    counts exact except for pairs whose exact distortion lies within 1e-6 of a
    bin edge or of eps (o.near_edge of them); max within 1e-5 and attained at
    the reported pair; mean within 1e-6.
    """
    assert g.pairs == o.pairs, (g.pairs, o.pairs)
    assert g.degenerate == o.degenerate, (g.degenerate, o.degenerate)
    slack = o.near_edge
    diff = int(np.abs(g.hist - o.hist).sum())
    assert diff <= 2 * slack, (diff, slack, g.hist, o.hist)
    assert abs(g.violations - o.violations) <= slack, (g.violations, o.violations, slack)
    assert abs(g.overflow - o.overflow) <= slack, (g.overflow, o.overflow, slack)
    assert int(g.hist.sum()) + g.overflow + g.degenerate == g.pairs
    assert abs(g.max - o.max) <= max_tol, (g.max, o.max)
    if o.pairs > o.degenerate:
        assert 0 <= g.argmax_i < g.argmax_j < X.shape[0]
        d_arg = pair_distortion(X, Y, [g.argmax_i], [g.argmax_j])[0]
        assert abs(d_arg - g.max) <= max_tol, (d_arg, g.max)
        assert abs(g.mean - o.mean) <= mean_tol, (g.mean, o.mean)
    assert g.max_err_bound <= 1e-5
