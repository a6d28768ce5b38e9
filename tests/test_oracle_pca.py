"""Pins for the oracle's centring, covariance and PCA (Sec. 2; Algorithm 1's P).

Pinned by data whose covariance spectrum and eigenvectors are known by
construction, by the 2-D closed form, and by the PCA distance bound of Sec. 3.
"""
import math

import numpy as np
import pytest

from oracle import adagio as O
from oracle.certificate import certificate


def _known_spectrum(rng, n, d, sig, shift=2.5):
    """X = H diag(sig) Q^T + c with H's columns orthonormal and orthogonal to 1."""
    G = np.concatenate([np.ones((n, 1)), rng.standard_normal((n, len(sig)))], axis=1)
    H, R = np.linalg.qr(G)
    H = H[:, 1:]                           # orthogonal to the all-ones column
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    Q = Q[:, :len(sig)]
    c = shift * rng.standard_normal(d)
    return H @ np.diag(sig) @ Q.T + c[None, :], Q


def test_known_spectrum_recovered():
    rng = np.random.default_rng(11)
    sig = np.array([9.0, 5.0, 3.0, 2.0, 1.0, 0.5])
    X, Q = _known_spectrum(rng, 200, 16, sig)
    pr = O.pca(X, 4)
    np.testing.assert_allclose(pr.theta[:6], sig ** 2, rtol=1e-11)
    assert np.all(np.abs(pr.theta[6:]) < 1e-10)
    for r in range(4):
        # eigenvector determined up to sign
        assert abs(abs(pr.P[r] @ Q[:, r]) - 1.0) < 1e-12
    np.testing.assert_allclose(pr.P @ pr.P.T, np.eye(4), atol=1e-13)


def test_two_dimensional_closed_form():
    # centred points +-a*u, +-b*v with u, v the rotation of e1, e2 by angle t
    a, b, t = 3.0, 1.0, 0.3
    u = np.array([math.cos(t), math.sin(t)])
    v = np.array([-math.sin(t), math.cos(t)])
    X = np.array([a * u, -a * u, b * v, -b * v]) + np.array([10.0, -4.0])
    pr = O.pca(X, 1)
    np.testing.assert_allclose(pr.theta, [2 * a * a, 2 * b * b], rtol=1e-13)
    # largest-magnitude entry made positive: u has cos t > sin t > 0
    np.testing.assert_allclose(pr.P[0], u, atol=1e-13)
    np.testing.assert_allclose(pr.mu, [10.0, -4.0], atol=1e-13)


def _low_rank(seed, n=120, d=10, r=3, noise=0.01):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((d, r)))
    z = rng.standard_normal((n, r)) * np.array([5.0, 4.0, 3.0])[None, :r]
    return z @ U.T + noise * rng.standard_normal((n, d)) + 2.0


def test_pca_distance_bound():
    """Sec. 3: PCA never expands and shrinks a pair by at most 2 sigma_{s+1}."""
    X = _low_rank(12)
    s = 3
    pr = O.pca(X, s)
    Y = O.embed(pr.P, X)
    sig_next = pr.sigma[s]
    n = X.shape[0]
    I, J = np.triu_indices(n, 1)
    dx = np.linalg.norm(X[I] - X[J], axis=1)
    dy = np.linalg.norm(Y[I] - Y[J], axis=1)
    assert np.all(dy <= dx * (1 + 1e-12))
    assert np.all(dx - dy <= 2 * sig_next * (1 + 1e-12))
    c = certificate(X, Y, eps=0.5, lo=0.0, hi=1.0)
    assert c.max <= 1.0
    assert c.max <= np.max(np.minimum(2 * sig_next / dx, 1.0)) + 1e-12


def test_wrong_direction_breaks_bound():
    """The bound above fails for the *bottom* eigenvectors (pin sensitivity)."""
    X = _low_rank(12)
    s = 3
    pr = O.pca(X, 10)
    P_bottom = pr.P[-s:]
    Y = O.embed(P_bottom, X)
    I, J = np.triu_indices(120, 1)
    dx = np.linalg.norm(X[I] - X[J], axis=1)
    dy = np.linalg.norm(Y[I] - Y[J], axis=1)
    assert np.any(dx - dy > 2 * pr.sigma[s])
