"""Pins of the warm-start network oracle: GELU closed forms and the
hand-written backward against central finite differences of the loss."""
import math

import numpy as np
import pytest

from oracle import warmstart as WS


def test_gelu_closed_forms():
    assert WS.gelu(np.array([0.0]))[0] == 0.0
    assert WS.gelu(np.array([10.0]))[0] == pytest.approx(10.0, rel=1e-15)
    assert WS.gelu(np.array([-10.0]))[0] == pytest.approx(0.0, abs=1e-20)
    # GELU(1) = Phi(1) = 0.5 (1 + erf(1/sqrt 2))
    assert WS.gelu(np.array([1.0]))[0] == pytest.approx(0.5 * (1 + math.erf(1 / math.sqrt(2))), rel=1e-15)
    a = np.linspace(-4, 4, 41)
    h = 1e-6
    np.testing.assert_allclose(WS.gelu_grad(a), (WS.gelu(a + h) - WS.gelu(a - h)) / (2 * h), rtol=1e-7, atol=1e-9)
    assert WS.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = WS.init_params(1)
    # two instances of different sizes, all four feature kinds
    seg = np.array([0] * 5 + [1] * 7)
    feats = rng.normal(size=(12, 4))
    extra = rng.uniform(1, 2, size=(2, 2))
    target = rng.normal(size=12)
    y, cache = WS.forward(P, feats, seg, extra)
    G = WS.backward(P, feats, seg, extra, target, cache)
    h = 1e-6
    for name in ("W1", "b1", "W2", "U", "b2", "w3", "b3"):
        flat = P[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for k in idx:
            old = flat[k]
            flat[k] = old + h
            fp = WS.mse(WS.forward(P, feats, seg, extra)[0], target)
            flat[k] = old - h
            fm = WS.mse(WS.forward(P, feats, seg, extra)[0], target)
            flat[k] = old
            assert G[name].reshape(-1)[k] == pytest.approx((fp - fm) / (2 * h), rel=1e-6, abs=1e-9)


def test_context_is_the_instance_mean():
    P = WS.init_params(2)
    rng = np.random.default_rng(3)
    feats = rng.normal(size=(6, 4))
    seg = np.array([0, 0, 0, 1, 1, 1])
    extra = np.ones((2, 2))
    # permuting points inside an instance permutes the outputs the same way
    y, _ = WS.forward(P, feats, seg, extra)
    perm = np.array([2, 0, 1, 5, 3, 4])
    y2, _ = WS.forward(P, feats[perm], seg, extra)
    np.testing.assert_allclose(y2, y[perm], rtol=1e-14)
