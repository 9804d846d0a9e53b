"""FP64 CPU oracle of the learned warm-start network (not part of the paper:
the "learned warm start" is an added component that predicts initial duals
for ASPOT).  TEST INFRASTRUCTURE ONLY: nothing in the CUDA library imports,
links or calls this module.

Network (per point, both clouds of one instance together):
    features  x_p = [coord_1, coord_2, N_side * weight_p / mass_side, side]   (side = +1 rows, -1 columns)
    a1 = W1 x_p + b1,             h1 = GELU(a1)                         (128)
    ctx_k = mean of h1 over the points of instance k                    (128)
    q_k  = U [ctx_k; |r|/s; |c|/s]                                       (128)
    a2 = W2 h1 + q_k + b2,         h2 = GELU(a2)                         (128)
    y_p = w3 . h2 + b3                                                   (1)
The target is gamma * u_i for a row point and gamma * v_j for a column point
(the duals ASPOT converged to); the loss is the mean squared error over all
points.  GELU(a) = a Phi(a) with the standard normal CDF Phi (erf form).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

H = 128
F = 4
E = 2            # extra context inputs: |r|_1 / s, |c|_1 / s


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / math.sqrt(2.0)))


def gelu_grad(a):
    return 0.5 * (1.0 + erf(a / math.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


def init_params(seed: int = 0) -> dict:
    g = np.random.default_rng(seed)
    return {
        "W1": g.normal(0.0, 1.0 / math.sqrt(F), (H, F)),
        "b1": np.zeros(H),
        "W2": g.normal(0.0, 1.0 / math.sqrt(H), (H, H)),
        "U": g.normal(0.0, 1.0 / math.sqrt(H + E), (H, H + E)),
        "b2": np.zeros(H),
        "w3": g.normal(0.0, 1.0 / math.sqrt(H), H),
        "b3": np.zeros(1),
    }


def segment_mean(h, seg, count):
    out = np.zeros((count, h.shape[1]))
    np.add.at(out, seg, h)
    n = np.bincount(seg, minlength=count).astype(np.float64)
    return out / n[:, None], n


def forward(P: dict, feats, seg, extra):
    """Returns y and the cache needed by backward."""
    count = extra.shape[0]
    a1 = feats @ P["W1"].T + P["b1"]
    h1 = gelu(a1)
    ctx, npts = segment_mean(h1, seg, count)
    cin = np.concatenate([ctx, extra], axis=1)
    q = cin @ P["U"].T
    a2 = h1 @ P["W2"].T + q[seg] + P["b2"]
    h2 = gelu(a2)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, dict(a1=a1, h1=h1, cin=cin, a2=a2, h2=h2, npts=npts)


def mse(y, target) -> float:
    d = y - target
    return float((d * d).mean())


def backward(P: dict, feats, seg, extra, target, cache) -> dict:
    """Gradients of the mean squared error by the chain rule, written out."""
    count = extra.shape[0]
    Np = feats.shape[0]
    dy = 2.0 * (cache["h2"] @ P["w3"] + P["b3"][0] - target) / Np
    g = {}
    g["w3"] = cache["h2"].T @ dy
    g["b3"] = np.array([dy.sum()])
    dh2 = np.outer(dy, P["w3"])
    da2 = dh2 * gelu_grad(cache["a2"])
    g["W2"] = da2.T @ cache["h1"]
    g["b2"] = da2.sum(axis=0)
    dq = np.zeros((count, H))
    np.add.at(dq, seg, da2)
    g["U"] = dq.T @ cache["cin"]
    dcin = dq @ P["U"]
    dctx = dcin[:, :H]
    dh1 = da2 @ P["W2"] + (dctx / cache["npts"][:, None])[seg]
    da1 = dh1 * gelu_grad(cache["a1"])
    g["W1"] = da1.T @ feats
    g["b1"] = da1.sum(axis=0)
    return g


def features(X, Y, r, c, s):
    """Per-point features and the per-instance extra inputs of one instance."""
    n, m = X.shape[0], Y.shape[0]
    fr = np.column_stack([X[:, 0], X[:, 1], n * r / r.sum(), np.ones(n)])
    fc = np.column_stack([Y[:, 0], Y[:, 1], m * c / c.sum(), -np.ones(m)])
    return np.vstack([fr, fc]), np.array([r.sum() / s, c.sum() / s])
