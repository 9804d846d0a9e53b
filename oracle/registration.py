"""FP64 CPU oracle of rigid point-cloud registration through POT (appendix,
"Point Cloud Registration"; experiment of Section 4.2).  TEST
INFRASTRUCTURE ONLY: nothing in the CUDA library imports, links or calls it.

Model: target cloud {x_i} (n points), source cloud {y_j} (m points), rigid
motion F(y) = R y + t applied to the source, and

    min_{R, t, pi}  sum_ij pi_ij |x_i - (R y_j + t)|^2,   pi in U(r, c, s).

Alternation (our reading of the appendix): with the motion fixed, pi is the
rounded ASPOT plan of the cost C_ij = |x_i - F(y_j)|^2; with pi fixed, the
motion is the weighted Procrustes solution

    u_x = sum_i (pi 1)_i x_i / |pi|_1,   u_y = sum_j (pi^T 1)_j y_j / |pi|_1,
    M = sum_ij pi_ij (x_i - u_x)(y_j - u_y)^T = U S V^T,
    R = U diag(1, 1, det(U V^T)) V^T,   t = u_x - R u_y.

The appendix prints R = V diag(1, 1, det(V U^T)) U^T for the SVD of the same
matrix; for the stated model F(y) = R y + t that is the transpose of the
minimiser (check: pi = identity matching and x = R0 y give M = R0 S with S
symmetric, so U V^T = R0), hence the form above (reading N19).  The source
moments are taken on the ORIGINAL source points, so each fit returns the
whole motion from the original cloud.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

from oracle import pot as O


def implicit_plan(C, gamma, f, g, p, q, kappa):
    """X_ij = exp(f_i + g_j - C_ij / gamma) + kappa p_i q_j (the rounded-plan form)."""
    return np.exp(np.asarray(f)[:, None] + np.asarray(g)[None, :] - np.asarray(C) / gamma) + \
        kappa * np.outer(p, q)


def rigid_fit(X, Y0, P):
    """Weighted Procrustes of the plan P (n x m) between target X (n x 3) and
    source Y0 (m x 3).  Returns (R, t, mass)."""
    X = np.asarray(X, dtype=np.float64)
    Y0 = np.asarray(Y0, dtype=np.float64)
    a = P.sum(axis=1)
    b = P.sum(axis=0)
    mass = float(P.sum())
    ux = (a[:, None] * X).sum(axis=0) / mass
    uy = (b[:, None] * Y0).sum(axis=0) / mass
    M = (X - ux).T @ P @ (Y0 - uy)
    U, S, Vt = np.linalg.svd(M)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt)) or 1.0])
    R = U @ D @ Vt
    t = ux - R @ uy
    return R, t, mass


def transform(Y0, R, t):
    return np.asarray(Y0) @ np.asarray(R).T + np.asarray(t)


def register(X, Y0, s, gamma0: float, anneal: float = 0.83, gamma_min: float = 0.0, eps: float = 1e-3,
             max_reg: int = 60, tol: float = 1e-5, max_iter: int = 20000):
    """The alternation above, uniform masses 1/n and 1/m, ASPOT (Algorithm 2)
    with gamma_k = max(gamma_min, gamma0 anneal^k) for registration k, the
    rounded plan, and the fit; stops when |R_k - R_{k-1}|_F + |t_k - t_{k-1}|
    < tol.  Returns (R, t, registrations, history of the transport cost)."""
    X = np.asarray(X, dtype=np.float64)
    Y0 = np.asarray(Y0, dtype=np.float64)
    n, m = X.shape[0], Y0.shape[0]
    r = np.full(n, 1.0 / n)
    c = np.full(m, 1.0 / m)
    R, t = np.eye(3), np.zeros(3)
    hist = []
    k = 0
    for k in range(1, max_reg + 1):
        gam = max(gamma_min, gamma0 * anneal ** (k - 1))
        Y = transform(Y0, R, t)
        C = O.sqeuclid_cost(X, Y, 1.0)
        sol = O.solve_aspot(C, r, c, s, eps, gam, max_iter=max_iter)
        P = sol.X
        hist.append(float((C * P).sum()))
        Rn, tn, _ = rigid_fit(X, Y0, P)
        delta = np.linalg.norm(Rn - R) + np.linalg.norm(tn - t)
        R, t = Rn, tn
        if delta < tol:
            break
    return R, t, k, hist


def rotation(axis, angle: float) -> np.ndarray:
    """Rodrigues' formula."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K
