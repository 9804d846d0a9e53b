"""FP64 CPU oracle of the learned warm-start network (not part of the paper:
the "learned warm start" is an added component that predicts initial duals
for ASPOT).  TEST INFRASTRUCTURE ONLY: nothing in the CUDA library imports,
links or calls this module.

Network (per point, both clouds of one instance together):
    features  x_p = [centred coordinates * sqrt(cost_scale), N_side * weight_p / mass_side, side,
                     soft minima of the cost to the other cloud's mass at temperatures
                     gamma, 4 gamma, 16 gamma]
              (side = +1 rows, -1 columns; F = d + 5 inputs)
    a1 = W1 x_p + b1,             h1 = GELU(a1)                         (128)
    ctx_k = mean of h1 over the points of instance k                    (128)
    q_k  = U [ctx_k; |r|/s; |c|/s]                                       (128)
    a2 = W2 h1 + q_k + b2,         h2 = GELU(a2)                         (128)
    y_p = w3 . h2 + b3                                                   (1)
The target is gamma log K (``targets``) for the duals (u, v, w) ASPOT
converged to, and the start from a prediction y is u = log r - softplus(y /
gamma), v = log c - softplus(y / gamma) (``warm_start``); the loss is the mean
squared error over all points.  GELU(a) = a Phi(a) with the standard normal CDF Phi (erf form).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

H = 128
EXTRA = 5        # per-point features besides the d coordinates
TEMPS = (1.0, 4.0, 16.0)   # soft-minimum temperatures, in units of gamma
F = 2 + EXTRA    # for d = 2
E = 2            # extra context inputs: |r|_1 / s, |c|_1 / s


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / math.sqrt(2.0)))


def gelu_grad(a):
    return 0.5 * (1.0 + erf(a / math.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


def init_params(seed: int = 0, d: int = 2) -> dict:
    g = np.random.default_rng(seed)
    F = d + EXTRA
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


def mse(y, target, weight=None) -> float:
    """(1/N) sum_p omega_p (y_p - target_p)^2 (omega = 1 when weight is None)."""
    d = y - target
    w = np.ones_like(d) if weight is None else np.asarray(weight, dtype=np.float64)
    return float((w * d * d).mean())


def backward(P: dict, feats, seg, extra, target, cache, weight=None) -> dict:
    """Gradients of the (weighted) mean squared error by the chain rule, written out."""
    count = extra.shape[0]
    Np = feats.shape[0]
    w = np.ones(Np) if weight is None else np.asarray(weight, dtype=np.float64)
    dy = 2.0 * w * (cache["h2"] @ P["w3"] + P["b3"][0] - target) / Np
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


def features(X, Y, r, c, s, gamma: float, cost_scale: float = 0.0):
    """Per-point features (rows first) and the per-instance extra inputs
    [|r|_1 / s, |c|_1 / s] of one instance.  Per point:
      centred coordinates * sqrt(cost_scale)           (mean over all n + m points)
      n r_i / |r|_1  or  m c_j / |c|_1
      +1 (row) or -1 (column)
      T log sum_j (c_j / |c|_1) exp(-C_ij / T)  for T = gamma, 4 gamma, 16 gamma
                                                 (row; a column uses r)
    with C = cost_scale |x - y|^2 and cost_scale 0 meaning 1 / max |x_i - y_j|^2
    (the normalisation of Section 4).  Masses below 1e-12 times their mean are
    floored inside the logarithm."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    n, m = X.shape[0], Y.shape[0]
    D = np.empty((n, m))
    for i in range(n):
        D[i] = ((X[i][None, :] - Y) ** 2).sum(axis=1)
    if cost_scale <= 0.0:
        mx = float(D.max())
        cost_scale = 1.0 / mx if mx > 0 else 1.0
    C = D * cost_scale
    lr = np.log(np.maximum(r, 1e-12 * r.sum() / n) / r.sum())
    lc = np.log(np.maximum(c, 1e-12 * c.sum() / m) / c.sum())
    soft_r = [np.array([T * gamma * _lse(lc - C[i] / (T * gamma)) for i in range(n)]) for T in TEMPS]
    soft_c = [np.array([T * gamma * _lse(lr - C[:, j] / (T * gamma)) for j in range(m)]) for T in TEMPS]
    mu = np.vstack([X, Y]).mean(axis=0)
    k = math.sqrt(cost_scale)
    fr = np.column_stack([(X - mu) * k, n * r / r.sum(), np.ones(n)] + soft_r)
    fc = np.column_stack([(Y - mu) * k, m * c / c.sum(), -np.ones(m)] + soft_c)
    return np.vstack([fr, fc]), np.array([r.sum() / s, c.sum() / s])


def _lse(a):
    mx = a.max()
    return mx + math.log(np.exp(a - mx).sum())


def adam_step(P: dict, G: dict, M: dict, V: dict, step: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8) -> None:
    """Adam (Kingma & Ba, 2015, Algorithm 1) in place: moment estimates,
    bias corrections 1 / (1 - b^step), update lr m_hat / (sqrt(v_hat) + eps)."""
    for k in P:
        M[k] = b1 * M[k] + (1.0 - b1) * G[k]
        V[k] = b2 * V[k] + (1.0 - b2) * G[k] * G[k]
        mh = M[k] / (1.0 - b1 ** step)
        vh = V[k] / (1.0 - b2 ** step)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)


def targets(C, gamma: float, u, v, w: float):
    """gamma log K_i = gamma (log sum_j B_ij - u_i) for rows and gamma (log
    sum_i B_ij - v_j) for columns, B = B(u, v, w) of Section 2: the log of the
    ratio of a point's transported mass to its slack e^{u_i} at the optimum,
    where (B1)_i + e^{u_i} = r_i gives u_i = log r_i - softplus(log K_i)."""
    from oracle import pot as O
    L = O.log_gibbs(C, gamma, u, v, w)
    lrow = np.array([_lse(L[i]) for i in range(L.shape[0])])
    lcol = np.array([_lse(L[:, j]) for j in range(L.shape[1])])
    return np.concatenate([gamma * (lrow - np.asarray(u)), gamma * (lcol - np.asarray(v))])


def target_weights(C, gamma: float, u, v, w: float):
    """Loss weights sigmoid(log K)^2 of the points (K from ``targets``): the
    squared factor by which an output error reaches the duals,
    du_i = sigmoid(y_i / gamma) dy_i / gamma at u_i = log r_i - softplus(y_i / gamma)."""
    lk = targets(C, gamma, u, v, w) / gamma
    sg = np.where(lk >= 0, 1.0 / (1.0 + np.exp(-np.abs(lk))), np.exp(-np.abs(lk)) / (1.0 + np.exp(-np.abs(lk))))
    return sg * sg


def softplus(x):
    x = np.asarray(x, dtype=np.float64)
    return np.where(x > 0, x + np.log1p(np.exp(-np.abs(x))), np.log1p(np.exp(-np.abs(x))))


def shift_step(C, gamma, r, c, s, u, v):
    """Exact minimiser of phi(u + a 1, v + b 1, w) over (a, b, w) for the dual of
    Section 2 (unsmoothed marginals): setting the three partial derivatives
    to zero gives e^(a+b+w) |B(u,v,0)|_1 = s, e^a sum e^u = |r| - s,
    e^b sum e^v = |c| - s (a = 0 when |r| = s, b = 0 when |c| = s)."""
    from oracle import pot as O
    L = O.log_gibbs(C, gamma, u, v, 0.0)
    ltot = _lse(L.reshape(-1))
    a = math.log(r.sum() - s) - _lse(np.asarray(u)) if r.sum() > s else 0.0
    b = math.log(c.sum() - s) - _lse(np.asarray(v)) if c.sum() > s else 0.0
    w = math.log(s) - ltot - a - b
    return np.asarray(u) + a, np.asarray(v) + b, w


def warm_start(P: dict, X, Y, r, c, s, gamma: float, cost_scale: float = 0.0):
    """The network's start for one problem: features, forward pass,
    u = log r - softplus(y / gamma), v = log c - softplus(y / gamma), then the
    shift step."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n, m = X.shape[0], Y.shape[0]
    f, e = features(X, Y, r, c, s, gamma, cost_scale)
    y, _ = forward(P, f, np.zeros(n + m, dtype=np.int64), e[None, :])
    br = np.log(np.maximum(r, 1e-12 * r.sum() / n))
    bc = np.log(np.maximum(c, 1e-12 * c.sum() / m))
    u, v = br - softplus(y[:n] / gamma), bc - softplus(y[n:] / gamma)
    D = np.array([((X[i][None, :] - Y) ** 2).sum(axis=1) for i in range(n)])
    cs = cost_scale if cost_scale > 0 else 1.0 / D.max()
    return shift_step(D * cs, gamma, np.asarray(r), np.asarray(c), s, u, v)


ORDER = ("W1", "b1", "W2", "U", "b2", "w3", "b3")


def unflatten(flat, d: int) -> dict:
    """Parameter dictionary from the flat layout W1[H][F], b1, W2[H][H], U[H][H+2], b2, w3, b3."""
    F = d + EXTRA
    shapes = {"W1": (H, F), "b1": (H,), "W2": (H, H), "U": (H, H + E), "b2": (H,), "w3": (H,), "b3": (1,)}
    out, o = {}, 0
    flat = np.asarray(flat, dtype=np.float64)
    for k in ORDER:
        size = int(np.prod(shapes[k]))
        out[k] = flat[o:o + size].reshape(shapes[k]).copy()
        o += size
    assert o == flat.size
    return out


def flatten(P: dict) -> np.ndarray:
    return np.concatenate([np.asarray(P[k], dtype=np.float64).reshape(-1) for k in ORDER])
