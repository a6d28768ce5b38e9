"""The benchmark's certified fit, checked against the FP64 oracle at full size.

The fit runs exactly as the benchmark times it: the 60 000 x 784
MNIST-shaped workload, eps = 0.1, FP16x3 tiles, the shipped dimension
predictor verified by the exhaustive certificate, PCA tolerance 1e-3.  Then
the oracle checks, on the GPU's own map A:

* the certificate of the returned map over all 1 799 970 000 pairs (Eq. 2,
  Eq. 3): histogram, overflow and violation counts exact except pairs within
  1e-6 of an edge or eps, maximum within 1e-5 and attained at its pair, mean
  within 1e-6;
* the embedding Y against the FP64 product X A^T (Algorithm 1), 1e-5 relative
  per row;
* the PCA part P = A[:s] (Sec. 2; randomized PCA, Sec. 4.5): orthonormal rows,
  and the energy it captures, tr(P C P^T), against the oracle's exact top-s
  eigenvalue sum;
* the JL part: A[s:] = S (I - P^T P) with the oracle's S (Algorithm 1).
"""
import os

import numpy as np
import pytest

from gpu_helpers import assert_cert_parity
from oracle import adagio as O
from oracle.certificate import certificate
from paper_1609_05388_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PREDICTOR = os.path.join(ROOT, "paper_1609_05388_gb300", "predictor_mnist_like.bin")


def test_headline_fit_against_oracle():
    from paper_1609_05388_gb300 import adagio as lib
    wl = synth.mnist_like(seed=1)
    X = wl.X
    n, d = X.shape
    Xd = torch.from_numpy(X).cuda()
    with lib.Context(0) as ctx:
        ctx.mlp_load(PREDICTOR)
        A, m, s, cert, rc = ctx.fit(Xd, eps=0.1, m_cap=d, seed=11, precision=lib.PREC_FP16X3,
                                    use_predictor=1, tol=1e-3)
        assert rc == 0 and cert.max <= 0.1 and s == m // 2
        Y = ctx.embed(A, Xd)
        torch.cuda.synchronize()
        Ah = A.cpu().numpy().astype(np.float64)
        Yh = Y.cpu().numpy()
    # the certificate of the returned map, every pair, by the oracle
    o = certificate(X, Yh, 0.1)
    assert o.pairs == n * (n - 1) // 2
    assert_cert_parity(cert, o, X, Yh)
    assert o.max <= 0.1 + 1e-5
    # Y = X A^T
    ref = X.astype(np.float64) @ Ah.T
    err = np.linalg.norm(Yh - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-30)
    assert err.max() <= 1e-5, err.max()
    # the PCA part: orthonormal rows capturing the top-s energy (the
    # Rayleigh-Ritz rotations run in FP32: about 6e-5 from orthonormality)
    P = Ah[:s]
    assert np.abs(P @ P.T - np.eye(s)).max() <= 1e-4
    pr = O.pca(X, s)
    _, Xc = O.centre(X)
    C = O.covariance(Xc)
    captured = np.trace(P @ C @ P.T)
    best = pr.theta[:s].sum()
    assert captured <= best * (1 + 1e-9)
    # the randomized PCA stops once every kept Ritz residual is below
    # 1e-3 theta_1; residuals alone bound no captured-energy deficit (the
    # eigenvalues near s = 210 are close together), so the check is at the
    # tolerance's scale; the deficit measured at this size is 6.5e-4
    assert captured >= (1 - 1e-3) * best, (captured, best)
    # the JL part: S (I - P^T P) with the oracle's S for the same seed
    S = O.jl_matrix(11, m - s, d)
    np.testing.assert_allclose(Ah[s:], S @ (np.eye(d) - P.T @ P), atol=2e-5)
