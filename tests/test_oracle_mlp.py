"""Pins of the predictor network's FP64 oracle (forward, backward, Adam) -- CPU only."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def test_gelu_identities():
    x = np.linspace(-6, 6, 101)
    # Phi(x) + Phi(-x) = 1  =>  GELU(x) - GELU(-x) = x
    np.testing.assert_allclose(M.gelu(x) - M.gelu(-x), x, atol=1e-14)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert M.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-15)
    # GELU(x) -> x for large x, -> 0 for very negative x
    assert M.gelu(np.array([10.0]))[0] == pytest.approx(10.0, abs=1e-12)
    assert abs(M.gelu(np.array([-10.0]))[0]) < 1e-20


def test_gelu_grad_matches_difference_quotient():
    x = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(M.gelu_grad(x), fd, atol=1e-8)


def _random_params(rng):
    p = {}
    for name, shape in M.SIZES:
        p[name] = rng.standard_normal(shape) * (0.2 if name.startswith("W") or name == "w3" else 0.1)
    return p


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    p = _random_params(rng)
    X = rng.standard_normal((7, M.IN))
    t = rng.standard_normal(7)
    loss, g = M.loss_and_grads(p, X, t)
    vec = M.pack(p)
    gvec = M.pack(g)
    idx = rng.choice(vec.size, 60, replace=False)
    idx = np.concatenate([idx, [M.NPARAM - 1, 0]])       # b3 and W1[0,0] too
    h = 1e-6
    for k in idx:
        vp, vm = vec.copy(), vec.copy()
        vp[k] += h
        vm[k] -= h
        lp, _ = M.loss_and_grads(M.unpack(vp), X, t)
        lm, _ = M.loss_and_grads(M.unpack(vm), X, t)
        fd = (lp - lm) / (2 * h)
        assert gvec[k] == pytest.approx(fd, rel=1e-5, abs=1e-9), k


def test_a_dropped_gelu_derivative_would_be_caught():
    rng = np.random.default_rng(1)
    p = _random_params(rng)
    X = rng.standard_normal((5, M.IN))
    t = rng.standard_normal(5)
    _, g = M.loss_and_grads(p, X, t)
    # rebuild W1's gradient without the GELU' factor: it must differ
    y, (X_, z1, h1, z2, h2) = M.forward(p, X)
    dy = 2 * (y - t) / 5
    dz2 = np.outer(dy, p["w3"]) * M.gelu_grad(z2)
    wrong = ((dz2 @ p["W2"])).T @ X_
    assert np.max(np.abs(wrong - g["W1"])) > 1e-3 * np.max(np.abs(g["W1"]))


def test_adam_first_step_closed_form():
    # first step: m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    vec = np.array([1.0, 1.0, 1.0, 1.0])
    new, m, v = M.adam_step(vec, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(new, vec - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_pack_roundtrip_and_bf16():
    rng = np.random.default_rng(2)
    vec = rng.standard_normal(M.NPARAM)
    np.testing.assert_array_equal(M.pack(M.unpack(vec)), vec)
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159], dtype=np.float32)
    r = M.bf16_round(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa wins (1.0)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert abs(r[3] - (-3.140625)) < 1e-12
