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


@pytest.mark.parametrize("weighted", [False, True])
def test_backward_matches_finite_differences(weighted):
    rng = np.random.default_rng(0)
    P = WS.init_params(1)
    # two instances of different sizes, all four feature kinds
    seg = np.array([0] * 5 + [1] * 7)
    feats = rng.normal(size=(12, 7))
    extra = rng.uniform(1, 2, size=(2, 2))
    target = rng.normal(size=12)
    wt = rng.uniform(0.0, 1.0, size=12) if weighted else None
    y, cache = WS.forward(P, feats, seg, extra)
    G = WS.backward(P, feats, seg, extra, target, cache, wt)
    h = 1e-6
    for name in ("W1", "b1", "W2", "U", "b2", "w3", "b3"):
        flat = P[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for k in idx:
            old = flat[k]
            flat[k] = old + h
            fp = WS.mse(WS.forward(P, feats, seg, extra)[0], target, wt)
            flat[k] = old - h
            fm = WS.mse(WS.forward(P, feats, seg, extra)[0], target, wt)
            flat[k] = old
            assert G[name].reshape(-1)[k] == pytest.approx((fp - fm) / (2 * h), rel=1e-6, abs=1e-9)


def test_context_is_the_instance_mean():
    P = WS.init_params(2)
    rng = np.random.default_rng(3)
    feats = rng.normal(size=(6, 7))
    seg = np.array([0, 0, 0, 1, 1, 1])
    extra = np.ones((2, 2))
    # permuting points inside an instance permutes the outputs the same way
    y, _ = WS.forward(P, feats, seg, extra)
    perm = np.array([2, 0, 1, 5, 3, 4])
    y2, _ = WS.forward(P, feats[perm], seg, extra)
    np.testing.assert_allclose(y2, y[perm], rtol=1e-14)


def test_features_hand_example_and_invariances():
    # two row points, one column point in 1-D: max |x - y|^2 = 4 (x=-1, y=1)
    X = np.array([[-1.0], [0.0]])
    Y = np.array([[1.0]])
    r = np.array([0.25, 0.75])
    c = np.array([1.5])
    g = 0.1
    f, e = WS.features(X, Y, r, c, s=0.5, gamma=g)
    # mean of all points = 0, sqrt(1/4) = 0.5; scaled costs C = [1, 1/4]
    np.testing.assert_allclose(f[:, 0], [-0.5, 0.0, 0.5])
    np.testing.assert_allclose(f[:, 1], [2 * 0.25, 2 * 0.75, 1.0])
    np.testing.assert_allclose(f[:, 2], [1, 1, -1])
    # one column: a row's soft minimum is its cost to that column at every temperature
    for t, T in enumerate((g, 4 * g, 16 * g)):
        np.testing.assert_allclose(f[:2, 3 + t], [-1.0, -0.25], rtol=1e-13)
        col = T * math.log(0.25 * math.exp(-1.0 / T) + 0.75 * math.exp(-0.25 / T))
        assert f[2, 3 + t] == pytest.approx(col, rel=1e-13)
    np.testing.assert_allclose(e, [2.0, 3.0])
    # translating both clouds or scaling them leaves the features unchanged
    rng = np.random.default_rng(0)
    X, Y = rng.normal(size=(7, 2)), rng.normal(size=(5, 2))
    r, c = rng.uniform(size=7), rng.uniform(size=5)
    f0, _ = WS.features(X, Y, r, c, 0.3, 0.05)
    f1, _ = WS.features(X + [3.0, -2.0], Y + [3.0, -2.0], r, c, 0.3, 0.05)
    f2, _ = WS.features(4.0 * X, 4.0 * Y, r, c, 0.3, 0.05)
    np.testing.assert_allclose(f1, f0, atol=1e-12)
    np.testing.assert_allclose(f2, f0, atol=1e-12)
    # the soft minimum lies between the smallest cost and the mass-weighted mean cost
    C = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    C = C / C.max()
    for t in range(3):
        sm = f0[:7, 4 + t]
        assert np.all(sm >= -C.max(axis=1) - 1e-12) and np.all(sm <= -C.min(axis=1) + 1e-12)
        assert np.all(sm >= -(C * (c / c.sum())).sum(axis=1) - 1e-12)   # Jensen
    # a higher temperature gives a softer (lower) minimum
    assert np.all(f0[:7, 5] <= f0[:7, 4] + 1e-12) and np.all(f0[:7, 6] <= f0[:7, 5] + 1e-12)
    # an explicit cost scale is used as given
    f3, _ = WS.features(X, Y, r, c, 0.3, 0.05, cost_scale=4.0)
    mu = np.vstack([X, Y]).mean(axis=0)
    np.testing.assert_allclose(f3[:7, :2], (X - mu) * 2.0)


def test_adam_first_step_is_lr_times_sign():
    # with zero moments the bias-corrected first step is lr * g / (|g| + eps)
    P = {"a": np.array([1.0, -2.0, 0.5])}
    G = {"a": np.array([3.0, -0.01, 0.0])}
    M = {"a": np.zeros(3)}
    V = {"a": np.zeros(3)}
    WS.adam_step(P, G, M, V, step=1, lr=0.1, eps=0.0 + 1e-12)
    np.testing.assert_allclose(P["a"], [0.9, -1.9, 0.5], atol=1e-9)


def test_flat_layout_round_trip():
    P = WS.init_params(4, d=3)
    flat = WS.flatten(P)
    assert flat.size == 128 * 8 + 128 + 128 * 128 + 128 * 130 + 128 + 128 + 1
    Q = WS.unflatten(flat, 3)
    for k in P:
        np.testing.assert_array_equal(Q[k], P[k])


def test_shift_step_zeroes_the_three_shift_derivatives():
    from oracle import pot as O
    rng = np.random.default_rng(4)
    n, m, g, s = 9, 7, 0.1, 0.6
    C = rng.uniform(size=(n, m))
    r, c = rng.uniform(0.5, 1.5, n), rng.uniform(0.5, 1.5, m)
    r, c = r / r.sum() * 1.1, c / c.sum() * 1.3
    u, v = rng.normal(-3, 1, n), rng.normal(-2, 1, m)
    u1, v1, w1 = WS.shift_step(C, g, r, c, s, u, v)
    B = np.exp(O.log_gibbs(C, g, u1, v1, w1))
    # d/da: sum_i dphi/du_i = |B| + sum e^u - |r|;  d/db likewise;  d/dw = |B| - s
    assert B.sum() == pytest.approx(s, rel=1e-12)
    assert B.sum() + np.exp(u1).sum() == pytest.approx(r.sum(), rel=1e-12)
    assert B.sum() + np.exp(v1).sum() == pytest.approx(c.sum(), rel=1e-12)
    # and phi does not increase against the plain w-step alone
    zw = O.Dual(u, v, math.log(s) - math.log(np.exp(O.log_gibbs(C, g, u, v, 0.0)).sum()))
    assert O.phi(C, g, r, c, s, O.Dual(u1, v1, w1)) <= O.phi(C, g, r, c, s, zw) + 1e-15
    # a point that already minimises phi along the shifts does not move
    u2, v2, w2 = WS.shift_step(C, g, r, c, s, u1, v1)
    np.testing.assert_allclose(u2, u1, atol=1e-12)
    np.testing.assert_allclose(v2, v1, atol=1e-12)
    assert w2 == pytest.approx(w1, abs=1e-12)


def test_targets_invert_the_start_at_the_optimum():
    """At the entropic optimum (B1)_i + e^{u_i} = r_i, so u_i = log r_i -
    softplus(log K_i): the start formula recovers the duals from the targets."""
    from oracle import pot as O
    import pot_workloads as W
    pb = W.tiny(3, n=6, m=5, mass_r=1.1, mass_c=1.4, s=0.8)
    C = np.asarray(pb.C, dtype=np.float64)
    res = O.aspot(C, pb.r, pb.c, pb.s, 1e-9, 0.1, max_iter=200000, smooth=False, stop_raw_eps=True)
    z = res.z
    t = WS.targets(C, 0.1, z.u, z.v, z.w)
    u = np.log(pb.r) - WS.softplus(t[:6] / 0.1)
    v = np.log(pb.c) - WS.softplus(t[6:] / 0.1)
    np.testing.assert_allclose(u, z.u, atol=1e-6)
    np.testing.assert_allclose(v, z.v, atol=1e-6)
    # softplus closed forms
    assert WS.softplus(0.0) == pytest.approx(math.log(2.0))
    assert WS.softplus(-50.0) == pytest.approx(math.exp(-50.0), rel=1e-12)
    assert WS.softplus(50.0) == pytest.approx(50.0, rel=1e-15)


def test_target_weights_are_the_squared_transported_fraction():
    """At the optimum sigmoid(log K_i) = (B1)_i / r_i: the fraction of r_i that
    is transported; its square is the weight."""
    from oracle import pot as O
    import pot_workloads as W
    pb = W.tiny(5, n=6, m=5, mass_r=1.1, mass_c=1.4, s=0.8)
    C = np.asarray(pb.C, dtype=np.float64)
    z = O.aspot(C, pb.r, pb.c, pb.s, 1e-9, 0.1, max_iter=200000, smooth=False, stop_raw_eps=True).z
    wts = WS.target_weights(C, 0.1, z.u, z.v, z.w)
    B = np.exp(O.log_gibbs(C, 0.1, z.u, z.v, z.w))
    np.testing.assert_allclose(np.sqrt(wts[:6]), B.sum(1) / pb.r, atol=1e-6)
    np.testing.assert_allclose(np.sqrt(wts[6:]), B.sum(0) / pb.c, atol=1e-6)
