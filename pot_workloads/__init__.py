"""Seeded synthetic inputs for partial optimal transport (POT) problems.

This module only draws inputs: point clouds, marginal weights, the mass
budget ``s`` and the entropic parameters of each workload.  It contains none
of the solver's arithmetic, so both the FP64 CPU oracle (``oracle/``) and the
CUDA library consume the very same problems.

Workloads (shapes follow the experiments of arXiv 2601.17196, whose own data
is not available; every input here is synthetic):

* ``small_dense``   n=m=256, 2-D, X ~ U[0,1]^2, Y ~ N((.5,.5), 0.1^2 I),
  squared-Euclidean cost divided by its max, |r|=1.0, |c|=1.2, s=0.8,
  gamma=0.05, eps=1e-3.  Stands in for the colour-transfer histograms
  (Section 4.1, n=800 colours, cost normalised by its max).
* ``dense_4096``    n=m=4096, 64-D, X ~ N(0,I), Y = 90% N(0,I) + 10% N(4*1,I),
  FP32 cost normalised to max 1, weights U[0.5,1.5] normalised to masses
  1.0 / 1.3, s=0.9, gamma in {0.1,0.03,0.01}, eps=1e-2.  Shaped like the
  synthetic scalability study (appendix, "ASPOT Synthetic Data Experiment":
  squared-Euclidean cost scaled to max 1, unequal masses).
* ``cloud_32k``     n=m=32768, 128-D BF16 points, 8-component Gaussian
  mixture (means ~ N(0,4I), unit covariance) with 5% uniform outliers in
  [-6,6]^128, uniform weights of masses 1.0 / 1.25, s=0.95, gamma=0.02,
  eps=1e-2.  The cost is never stored; it is normalised by its max.
* ``batch_3d``      512 instances, n_k,m_k ~ U{64..2048}, 3-D points in
  [0,1]^3, |r|=1, |c| ~ U[1,1.5], s_k ~ U[0.5,0.95], gamma=0.05, eps=1e-3.
  Stands in for the 3-D point-cloud registration problems (Section 4.2).
* ``scaling_e4``    the appendix's scalability study: two random non-negative
  weight vectors of masses 5 and 3 on n points each, squared-Euclidean cost
  between the points scaled to max 1, s = 0.2 min(5, 3) = 0.6, gamma = 1e-3;
  the points are not specified there, so they are drawn U[0,1]^2 here.
* ``mix_2d``        n=m=1024, 2-D mixtures of 2-6 Gaussians, masses
  U[1,1.5], s ~ U[0.6,0.95] (below both masses), gamma=0.02,
  eps=1e-3 (learned warm-start data).

Every generator takes ``n`` / ``m`` overrides so that tests can draw the same
recipe at sizes the oracle finishes in seconds.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """One POT instance.  Arrays are numpy; ``C`` is the dense FP32 cost
    (row-major n x m) when the workload stores it, else None and the cost is
    the squared Euclidean distance between rows of ``X`` and ``Y`` times
    ``cost_scale`` (0 means "divide by the maximum distance")."""

    name: str
    r: np.ndarray            # float64 [n]
    c: np.ndarray            # float64 [m]
    s: float
    gamma: float
    eps: float
    C: Optional[np.ndarray] = None      # float32 [n, m]
    X: Optional[np.ndarray] = None      # float64 [n, d] exact point values
    Y: Optional[np.ndarray] = None      # float64 [m, d]
    X_bf16: Optional[np.ndarray] = None  # uint16 bit patterns of X (BF16)
    Y_bf16: Optional[np.ndarray] = None
    cost_scale: float = 0.0

    @property
    def n(self) -> int:
        return int(self.r.shape[0])

    @property
    def m(self) -> int:
        return int(self.c.shape[0])


def to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round to nearest, ties to even) and
    return the 16-bit patterns as uint16."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = (bits + 0x7FFF + lsb) >> 16
    return rounded.astype(np.uint16)


def from_bf16_bits(b: np.ndarray) -> np.ndarray:
    """Exact float64 values of bfloat16 bit patterns."""
    u = b.astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def _sqdist(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Plain squared Euclidean distances, FP64, used to build dense inputs."""
    D = (X * X).sum(1)[:, None] + (Y * Y).sum(1)[None, :] - 2.0 * (X @ Y.T)
    return np.maximum(D, 0.0)


def _normalised_f32(D: np.ndarray) -> np.ndarray:
    return (D / D.max()).astype(np.float32)


def small_dense(seed: int = 0, n: int = 256, m: Optional[int] = None,
                gamma: float = 0.05, eps: float = 1e-3) -> Problem:
    m = n if m is None else m
    g = np.random.default_rng(seed)
    X = g.uniform(0.0, 1.0, size=(n, 2))
    Y = g.normal(0.5, 0.1, size=(m, 2))
    C = _normalised_f32(_sqdist(X, Y))
    r = np.full(n, 1.0 / n)
    c = np.full(m, 1.2 / m)
    return Problem("small_dense", r, c, 0.8, gamma, eps, C=C, X=X, Y=Y, cost_scale=1.0)


def dense_4096(seed: int = 0, n: int = 4096, m: Optional[int] = None, d: int = 64,
               gamma: float = 0.03, eps: float = 1e-2) -> Problem:
    m = n if m is None else m
    g = np.random.default_rng(seed)
    X = g.normal(0.0, 1.0, size=(n, d))
    Y = g.normal(0.0, 1.0, size=(m, d))
    n_out = int(round(0.1 * m))
    Y[:n_out] += 4.0
    g.shuffle(Y, axis=0)
    C = _normalised_f32(_sqdist(X, Y))
    wr = g.uniform(0.5, 1.5, size=n)
    wc = g.uniform(0.5, 1.5, size=m)
    r = wr / wr.sum() * 1.0
    c = wc / wc.sum() * 1.3
    return Problem("dense_4096", r, c, 0.9, gamma, eps, C=C, X=X, Y=Y, cost_scale=1.0)


def _gmm_cloud(g: np.random.Generator, npts: int, means: np.ndarray,
               outlier_frac: float, box: float) -> np.ndarray:
    k, d = means.shape
    lab = g.integers(0, k, size=npts)
    P = means[lab] + g.normal(0.0, 1.0, size=(npts, d))
    n_out = int(round(outlier_frac * npts))
    P[:n_out] = g.uniform(-box, box, size=(n_out, d))
    g.shuffle(P, axis=0)
    return P


def cloud_32k(seed: int = 0, n: int = 32768, m: Optional[int] = None, d: int = 128,
              gamma: float = 0.02, eps: float = 1e-2) -> Problem:
    m = n if m is None else m
    g = np.random.default_rng(seed)
    means = g.normal(0.0, 2.0, size=(8, d))      # N(0, 4 I)
    Xf = _gmm_cloud(g, n, means, 0.05, 6.0)
    Yf = _gmm_cloud(g, m, means, 0.05, 6.0)
    Xb, Yb = to_bf16_bits(Xf), to_bf16_bits(Yf)
    X, Y = from_bf16_bits(Xb), from_bf16_bits(Yb)
    r = np.full(n, 1.0 / n)
    c = np.full(m, 1.25 / m)
    return Problem("cloud_32k", r, c, 0.95, gamma, eps, X=X, Y=Y,
                   X_bf16=Xb, Y_bf16=Yb, cost_scale=0.0)


def batch_3d(seed: int = 0, count: int = 512, nmin: int = 64, nmax: int = 2048,
             gamma: float = 0.05, eps: float = 1e-3) -> list:
    """``count`` independent instances with uneven sizes.  Points are FP32
    values (stored exactly in float64)."""
    g = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(g.integers(nmin, nmax + 1))
        m = int(g.integers(nmin, nmax + 1))
        X = g.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32).astype(np.float64)
        Y = g.uniform(0.0, 1.0, size=(m, 3)).astype(np.float32).astype(np.float64)
        ratio = float(g.uniform(1.0, 1.5))
        s = float(g.uniform(0.5, 0.95))
        r = np.full(n, 1.0 / n)
        c = np.full(m, ratio / m)
        out.append(Problem(f"batch_3d[{k}]", r, c, s, gamma, eps, X=X, Y=Y, cost_scale=0.0))
    return out


def mix_2d(seed: int = 0, n: int = 1024, m: Optional[int] = None,
           gamma: float = 0.02, eps: float = 1e-3) -> Problem:
    m = n if m is None else m
    g = np.random.default_rng(seed)

    def cloud(npts):
        k = int(g.integers(2, 7))
        means = g.uniform(-1.0, 1.0, size=(k, 2))
        scales = g.uniform(0.05, 0.3, size=k)
        w = g.dirichlet(np.ones(k))
        lab = g.choice(k, size=npts, p=w)
        return (means[lab] + g.normal(size=(npts, 2)) * scales[lab][:, None]).astype(np.float32).astype(np.float64)

    X, Y = cloud(n), cloud(m)
    mr, mc = float(g.uniform(1.0, 1.5)), float(g.uniform(1.0, 1.5))
    wr, wc = g.uniform(0.5, 1.5, size=n), g.uniform(0.5, 1.5, size=m)
    r = wr / wr.sum() * mr
    c = wc / wc.sum() * mc
    s = float(g.uniform(0.6, 0.95))          # both masses are >= 1 > s
    return Problem("mix_2d", r, c, s, gamma, eps, X=X, Y=Y, cost_scale=0.0)


def scaling_e4(seed: int = 0, n: int = 1000, gamma: float = 1e-3, eps: float = 1e-7) -> Problem:
    g = np.random.default_rng(seed)
    X = g.uniform(0.0, 1.0, size=(n, 2))
    Y = g.uniform(0.0, 1.0, size=(n, 2))
    C = _normalised_f32(_sqdist(X, Y))
    wr, wc = g.uniform(0.0, 1.0, size=n), g.uniform(0.0, 1.0, size=n)
    r = wr / wr.sum() * 5.0
    c = wc / wc.sum() * 3.0
    return Problem("scaling_e4", r, c, 0.6, gamma, eps, C=C, X=X, Y=Y, cost_scale=1.0)


def tiny(seed: int = 0, n: int = 5, m: int = 6, d: int = 2, mass_r: float = 1.0,
         mass_c: float = 1.3, s: float = 0.7, gamma: float = 0.05, eps: float = 1e-2,
         uniform: bool = False) -> Problem:
    """Tiny dense instance for exact-LP and brute-force checks."""
    g = np.random.default_rng(seed)
    X = g.uniform(0.0, 1.0, size=(n, d))
    Y = g.uniform(0.0, 1.0, size=(m, d))
    C = _normalised_f32(_sqdist(X, Y))
    if uniform:
        r = np.full(n, mass_r / n)
        c = np.full(m, mass_c / m)
    else:
        wr, wc = g.uniform(0.5, 1.5, size=n), g.uniform(0.5, 1.5, size=m)
        r = wr / wr.sum() * mass_r
        c = wc / wc.sum() * mass_c
    return Problem("tiny", r, c, s, gamma, eps, C=C, X=X, Y=Y, cost_scale=1.0)


# --------------------------------------------------------------------------
# Warm-start network inputs (random numbers only; the network's arithmetic
# lives in the oracle and in the CUDA library)
# --------------------------------------------------------------------------

WS_HIDDEN = 128


def ws_params(d: int = 2, seed: int = 0, bias_scale: float = 0.1) -> np.ndarray:
    """Flat FP32 parameter vector in the library's layout W1[H][F], b1[H],
    W2[H][H], U[H][H+2], b2[H], w3[H], b3[1] (F = d + 5): weights
    N(0, 1/fan_in), biases N(0, bias_scale^2) so that every block is
    exercised by a gradient check."""
    g = np.random.default_rng(seed)
    H, F = WS_HIDDEN, d + 5
    parts = [g.normal(0, 1 / np.sqrt(F), H * F), g.normal(0, bias_scale, H),
             g.normal(0, 1 / np.sqrt(H), H * H), g.normal(0, 1 / np.sqrt(H + 2), H * (H + 2)),
             g.normal(0, bias_scale, H), g.normal(0, 1 / np.sqrt(H), H), g.normal(0, bias_scale, 1)]
    return np.concatenate(parts).astype(np.float32)


def ws_batch(sizes, d: int = 2, seed: int = 0):
    """Random feature sets: per instance `size` points with F = d + 5 features
    (coordinates N(0, 0.3^2), weight ratio U[0.5, 1.5], side +-1, three soft
    minima U[-0.5, 0]), extra inputs U[1, 2] and targets N(-0.05, 0.05^2).
    Returns (feats [N][F] f32, extra [K][2] f32, target [N] f32, off [K+1] int64)."""
    g = np.random.default_rng(seed)
    F = d + 5
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    N = int(off[-1])
    feats = np.empty((N, F), dtype=np.float32)
    feats[:, :d] = g.normal(0, 0.3, size=(N, d))
    feats[:, d] = g.uniform(0.5, 1.5, size=N)
    feats[:, d + 1] = np.where(g.uniform(size=N) < 0.5, 1.0, -1.0)
    feats[:, d + 2:] = g.uniform(-0.5, 0.0, size=(N, 3))
    extra = g.uniform(1.0, 2.0, size=(len(sizes), 2)).astype(np.float32)
    target = g.normal(-0.05, 0.05, size=N).astype(np.float32)
    return feats, extra, target, off


def ws_weights(n: int, seed: int = 0) -> np.ndarray:
    """Random loss weights U[0, 1] (FP32) for weighted-loss checks."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=n).astype(np.float32)


def registration_3d(seed: int = 0, n: int = 1024, frac: float = 0.5, max_angle: float = 0.5,
                    max_shift: float = 0.1, noise: float = 0.0):
    """A target cloud and a misaligned partial source (stand-in for the 3-D
    registration clouds of Section 4.2): the target is n points on three
    random ellipsoid surfaces in [0.15, 0.85]^3; the source is a fraction
    `frac` of it (one contiguous half-space side, so the overlap is partial),
    moved by a random rotation of angle <= max_angle about a random axis and a
    shift of norm <= max_shift, plus Gaussian noise.  Returns
    (X [n,3], Y0 [m,3], R_true, t_true) with R_true Y0 + t_true = the chosen
    target points (before noise)."""
    g = np.random.default_rng(seed)
    k = 3
    centres = g.uniform(0.35, 0.65, size=(k, 3))
    radii = g.uniform(0.08, 0.2, size=(k, 3))
    lab = g.integers(0, k, size=n)
    dirs = g.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    X = centres[lab] + dirs * radii[lab]
    normal = g.normal(size=3)
    normal /= np.linalg.norm(normal)
    proj = (X - X.mean(axis=0)) @ normal
    keep = np.argsort(proj)[: int(round(frac * n))]
    axis = g.normal(size=3)
    axis /= np.linalg.norm(axis)
    angle = g.uniform(0.3, 1.0) * max_angle
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    R_true = np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K
    shift = g.normal(size=3)
    t_true = shift / np.linalg.norm(shift) * g.uniform(0.3, 1.0) * max_shift
    # R_true y0 + t_true = x  =>  y0 = R_true^T (x - t_true)
    Y0 = (X[keep] - t_true) @ R_true
    if noise > 0:
        Y0 = Y0 + g.normal(scale=noise, size=Y0.shape)
    X = X.astype(np.float32).astype(np.float64)
    Y0 = Y0.astype(np.float32).astype(np.float64)
    return X, Y0, R_true, t_true


def plan_params(n: int, m: int, seed: int = 0, gamma: float = 0.05):
    """Random implicit-plan parameters (f, g, p, q, kappa) for checks of plan
    moment kernels: f, g ~ U[-2, 0] + log(1/n), p, q ~ U[0, 1/n], kappa
    U[0.5, 2]."""
    g = np.random.default_rng(seed)
    f = g.uniform(-2.0, 0.0, size=n) + np.log(1.0 / n)
    gg = g.uniform(-2.0, 0.0, size=m) + np.log(1.0 / m)
    p = g.uniform(0.0, 1.0 / n, size=n)
    q = g.uniform(0.0, 1.0 / m, size=m)
    return f, gg, p, q, float(g.uniform(0.5, 2.0))
