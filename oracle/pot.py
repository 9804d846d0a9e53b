"""FP64 CPU oracle for entropic Partial Optimal Transport (arXiv 2601.17196).

TEST INFRASTRUCTURE ONLY.  Nothing in the CUDA library imports, links or
calls this module; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.  It shares no code with the GPU
path: it is a plain, slow, obviously correct restatement of the paper in
numpy float64, written so that each function can be checked against the
paper by eye.

Notation (Section 2.1): marginals r in R^n_+, c in R^m_+, budget
s <= min(|r|_1, |c|_1), cost C in R^{n x m}_+, entropic parameter gamma,
dual point z = (u, v, w) with u in R^n, v in R^m, w in R, and

    B(z)_ij = exp(-C_ij / gamma + u_i + v_j + w)                 (Eq. dual)
    phi(z)  = |B(z)|_1 + sum_i e^{u_i} + sum_j e^{v_j}
              - <u, r> - <v, c> - w s                             (Eq. dual)

The paper states everything with m = n; every function here allows m != n
(the point-cloud appendix already uses two sizes).

Readings of passages that are silent or ambiguous:
  * N2  the zero start "0_{n+1}" of Algorithm 2 is the zero dual point
        (u, v, w) = 0 in R^{n+m+1}.
  * N3  inside the loop every marginal is the smoothed one (r~, c~): in the
        Greenkhorn steps, the gradient, phi, E(t) and the step size; the
        rounding uses the caller's original r, c, s.
  * N4  E_t is E(z^t) measured after the argmin, tested at the end of each
        iteration; the primal is formed from that same z^t.
  * N5  the mass guards of Algorithm 2's setup shrink the smoothing
        coefficient; the stop threshold stays eps / (8 max C).  A guard that
        yields 0 (|r|_1 == s) switches smoothing off.
  * N6  gamma is an input; gamma <= 0 selects the default eps / (4 log n)
        with n = max(n, m).
  * N8  the argmin keeps the Greenkhorn point z^ only when phi(z^) < phi(z_check)
        strictly.
  * N10 the gradient step is 1/(L theta_t) with L = 3 (|r~|_1+|c~|_1-s)/gamma.
  * N11 the dummy cost of the feasible Sinkhorn baseline is A = 8 max C / eps.
  * N13 the Sinkhorn baseline uses Algorithm 2's setup (gamma, threshold and
        smoothing), as the experiments of Section 4.1 state.
  * N17 with a zero dummy mass (balanced case) the dummy row / column is
        dropped.
  * R1-R4 ROUND-POT is cited but not written out; ``round_pot`` below is the
        reading used (row scale-down, column scale-down, then either a
        uniform scale to mass s or a rank-one fill of the slack).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np


# --------------------------------------------------------------------------
# Costs
# --------------------------------------------------------------------------

def sqeuclid_cost(X: np.ndarray, Y: np.ndarray, cost_scale: float = 0.0) -> np.ndarray:
    """C_ij = cost_scale * sum_k (x_ik - y_jk)^2, row by row from the
    definition.  cost_scale == 0 divides by the largest entry (the
    normalisation "C / max C" used by every experiment of Section 4)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    C = np.empty((X.shape[0], Y.shape[0]))
    for i in range(X.shape[0]):
        diff = X[i][None, :] - Y
        C[i] = (diff * diff).sum(axis=1)
    if cost_scale == 0.0:
        cost_scale = 1.0 / C.max()
    return C * cost_scale


def sqeuclid_rows(X: np.ndarray, Y: np.ndarray, rows: Sequence[int], cost_scale: float) -> np.ndarray:
    """Selected rows of the scaled squared-Euclidean cost (for sampled checks
    at sizes where the full matrix is too large)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    out = np.empty((len(rows), Y.shape[0]))
    for k, i in enumerate(rows):
        diff = X[i][None, :] - Y
        out[k] = (diff * diff).sum(axis=1) * cost_scale
    return out


# --------------------------------------------------------------------------
# Log-sum-exp and the Gibbs matrix B(z)
# --------------------------------------------------------------------------

def logsumexp(a: np.ndarray, axis=None) -> np.ndarray:
    """log(sum(exp(a))) with the usual max shift; -inf for all -inf input."""
    a = np.asarray(a, dtype=np.float64)
    mx = np.max(a, axis=axis, keepdims=True)
    mx = np.where(np.isfinite(mx), mx, 0.0)
    out = np.log(np.sum(np.exp(a - mx), axis=axis, keepdims=True)) + mx
    if axis is None:
        return float(out.reshape(()))
    return np.squeeze(out, axis=axis)


def log_gibbs(C: np.ndarray, gamma: float, u, v, w) -> np.ndarray:
    """log B(z)_ij = -C_ij/gamma + u_i + v_j + w (Eq. dual)."""
    return -C / gamma + np.asarray(u)[:, None] + np.asarray(v)[None, :] + w


def row_sums(C, gamma, u, v, w) -> np.ndarray:
    """r(B(z)) = B(z) 1_m."""
    return np.exp(logsumexp(log_gibbs(C, gamma, u, v, w), axis=1))


def col_sums(C, gamma, u, v, w) -> np.ndarray:
    """c(B(z)) = B(z)^T 1_n."""
    return np.exp(logsumexp(log_gibbs(C, gamma, u, v, w), axis=0))


def total_mass(C, gamma, u, v, w) -> float:
    """|B(z)|_1 = 1_n^T B(z) 1_m."""
    return math.exp(logsumexp(log_gibbs(C, gamma, u, v, w)))


def rho(a, b):
    """rho(a, b) = b - a + a log(a/b) (Section 2.1, notation)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return b - a + a * np.log(a / b)


def entropy(x) -> float:
    """H(x) = -<x, log x> (Section 2.1, notation)."""
    x = np.asarray(x, dtype=np.float64)
    x = x[x > 0]
    return float(-(x * np.log(x)).sum())


# --------------------------------------------------------------------------
# Dual objective, gradient, feasibility error, Greenkhorn step
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Dual:
    u: np.ndarray
    v: np.ndarray
    w: float

    def copy(self) -> "Dual":
        return Dual(self.u.copy(), self.v.copy(), float(self.w))

    def axpby(self, a: float, other: "Dual", b: float) -> "Dual":
        """a * self + b * other."""
        return Dual(a * self.u + b * other.u, a * self.v + b * other.v, a * self.w + b * other.w)

    def flat(self) -> np.ndarray:
        return np.concatenate([self.u, self.v, [self.w]])

    @staticmethod
    def zeros(n: int, m: int) -> "Dual":
        return Dual(np.zeros(n), np.zeros(m), 0.0)


def phi(C, gamma, r, c, s, z: Dual) -> float:
    """Dual objective phi(z) of entropic POT (Eq. dual)."""
    return (total_mass(C, gamma, z.u, z.v, z.w) + np.exp(z.u).sum() + np.exp(z.v).sum()
            - z.u @ r - z.v @ c - z.w * s)


def grad_phi(C, gamma, r, c, s, z: Dual) -> Dual:
    """Gradient of phi: (r(B)+e^u-r, c(B)+e^v-c, |B|_1-s)."""
    L = log_gibbs(C, gamma, z.u, z.v, z.w)
    rB = np.exp(logsumexp(L, axis=1))
    cB = np.exp(logsumexp(L, axis=0))
    tot = math.exp(logsumexp(L))
    return Dual(rB + np.exp(z.u) - r, cB + np.exp(z.v) - c, tot - s)


def feas_error(C, gamma, r, c, s, z: Dual) -> float:
    """E = |1^T B 1 - s| + |B 1 + p - r|_1 + |B^T 1 + q - c|_1 with the slack
    estimates p = e^u, q = e^v (Section 3.1, the monitored error E(t))."""
    L = log_gibbs(C, gamma, z.u, z.v, z.w)
    rB = np.exp(logsumexp(L, axis=1))
    cB = np.exp(logsumexp(L, axis=0))
    tot = math.exp(logsumexp(L))
    return float(abs(tot - s) + np.abs(rB + np.exp(z.u) - r).sum() + np.abs(cB + np.exp(z.v) - c).sum())


def block_decreases(C, gamma, r, c, s, z: Dual) -> np.ndarray:
    """Exact decrease of phi for each of the three block steps at z
    (proof of Theorem 3): sum_i rho(r_i, r_i(B)+e^{u_i}),
    sum_j rho(c_j, c_j(B)+e^{v_j}), rho(s, |B|_1)."""
    L = log_gibbs(C, gamma, z.u, z.v, z.w)
    rB = np.exp(logsumexp(L, axis=1))
    cB = np.exp(logsumexp(L, axis=0))
    tot = math.exp(logsumexp(L))
    return np.array([rho(r, rB + np.exp(z.u)).sum(), rho(c, cB + np.exp(z.v)).sum(), float(rho(s, tot))])


def greenkhorn_step(C, gamma, r, c, s, z: Dual, k: int) -> Dual:
    """Algorithm 1 (Greenkhorn step) for block k: 0 -> u, 1 -> v, 2 -> w.

    u <- u + log r - log(r(B) + e^u); v likewise with columns;
    w <- w + log s - log |B|_1.  The sums r(B) + e^u are formed in the log
    domain (log(r(B)_i + e^{u_i}) = logaddexp(log r(B)_i, u_i))."""
    L = log_gibbs(C, gamma, z.u, z.v, z.w)
    out = z.copy()
    if k == 0:
        out.u = z.u + np.log(r) - np.logaddexp(logsumexp(L, axis=1), z.u)
    elif k == 1:
        out.v = z.v + np.log(c) - np.logaddexp(logsumexp(L, axis=0), z.v)
    elif k == 2:
        out.w = z.w + math.log(s) - logsumexp(L)
    else:
        raise ValueError("block index must be 0, 1 or 2")
    return out


# --------------------------------------------------------------------------
# Algorithm 2, setup ("Approximating POT")
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Setup:
    gamma: float
    eps_stop: float      # stop threshold eps~ = eps / (8 max C)
    eps_smooth: float    # guarded coefficient used for the smoothing
    r_t: np.ndarray      # smoothed marginals r~, c~
    c_t: np.ndarray
    T: float             # |r~|_1 + |c~|_1 - s
    L: float             # 3 T / gamma


def approx_setup(r, c, s, eps, cmax, gamma: Optional[float] = None, smooth: bool = True) -> Setup:
    """Setup of Algorithm 2: gamma = eps/(4 log n), eps~ = eps/(8 |C|_max),
    the two mass guards eps~ <- min(eps~, 8(|r|-s)/(|r|-1)) when |r| > 1 (and
    the same for c), and the smoothing r~ = (1-eps~/8) r + eps~/(8n) 1."""
    r = np.asarray(r, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    n, m = r.shape[0], c.shape[0]
    if gamma is None or gamma <= 0:
        gamma = eps / (4.0 * math.log(max(n, m)))
    eps_stop = eps / (8.0 * cmax)
    e = eps_stop
    mr, mc = r.sum(), c.sum()
    if mr > 1.0:
        e = min(e, 8.0 * (mr - s) / (mr - 1.0))
    if mc > 1.0:
        e = min(e, 8.0 * (mc - s) / (mc - 1.0))
    if not smooth or e <= 0.0:
        e = 0.0
    r_t = (1.0 - e / 8.0) * r + e / (8.0 * n)
    c_t = (1.0 - e / 8.0) * c + e / (8.0 * m)
    T = r_t.sum() + c_t.sum() - s
    return Setup(gamma, eps_stop, e, r_t, c_t, T, 3.0 * T / gamma)


def theta_next(theta: float) -> float:
    """theta_{t+1} = theta_t (sqrt(theta_t^2 + 4) - theta_t) / 2 (Algorithm 2)."""
    return theta * (math.sqrt(theta * theta + 4.0) - theta) / 2.0


def dual_radius(r, c, s, gamma, cinf) -> float:
    """Bound R on the optimal duals (Eq. R, from the cited feasible-Sinkhorn
    analysis)."""
    mx = max(float(np.sum(r)), float(np.sum(c)))
    return cinf * mx / (gamma * (mx - s)) - math.log(min(float(np.min(r)), float(np.min(c))))


# --------------------------------------------------------------------------
# Algorithm 2: ASPOT
# --------------------------------------------------------------------------

@dataclasses.dataclass
class AspotTrace:
    k: List[int] = dataclasses.field(default_factory=list)          # block of iteration t
    k2: List[int] = dataclasses.field(default_factory=list)         # block of the step at z^t
    dec: List[tuple] = dataclasses.field(default_factory=list)      # greedy: block decreases at z_grave, at z^t
    took_hat: List[bool] = dataclasses.field(default_factory=list)  # argmin picked z^
    E: List[float] = dataclasses.field(default_factory=list)
    theta: List[float] = dataclasses.field(default_factory=list)
    phi_grave: List[float] = dataclasses.field(default_factory=list)
    phi_hat: List[float] = dataclasses.field(default_factory=list)
    phi_z: List[float] = dataclasses.field(default_factory=list)
    phi_check_next: List[float] = dataclasses.field(default_factory=list)
    z_tilde: List[np.ndarray] = dataclasses.field(default_factory=list)


@dataclasses.dataclass
class SolveResult:
    z: Dual              # final dual point z^t
    iters: int
    E: float
    setup: Setup
    converged: bool
    trace: Optional[AspotTrace] = None
    z_check: Optional[Dual] = None


def _choose_block(rule: str, t: int, C, gamma, r, c, s, z: Dual) -> int:
    if rule == "cyclic":
        return t % 3
    if rule == "greedy":
        return int(np.argmax(block_decreases(C, gamma, r, c, s, z)))
    raise ValueError(rule)


def aspot(C, r, c, s, eps, gamma: Optional[float] = None, max_iter: int = 10000,
          block_rule: str = "cyclic", stop_raw_eps: bool = False, smooth: bool = True,
          z0: Optional[Dual] = None, forced_hat: Optional[Sequence[bool]] = None,
          record: bool = False, cmax: Optional[float] = None, no_stop: bool = False,
          forced_blocks: Optional[Sequence[tuple]] = None) -> SolveResult:
    """Algorithm 2 (Accelerated Sinkhorn for POT), main loop.

    Per iteration t (theta_0 = 1, z~^0 = z_check^0 = 0 or the warm start):
      z_bar  = (1-theta) z_check + theta z~                      extrapolation
      z~'    = z_bar - grad phi(z_bar) / (L theta)               gradient step
      z_grave= z_bar + theta (z~' - z~)                          coupling
      z^     = Greenkhorn_k(z_grave)
      z^t    = argmin{phi(z_check), phi(z^)}
      E_t    = E(z^t)
      z_check= Greenkhorn_k(z^t)
      theta  = theta (sqrt(theta^2+4) - theta)/2
    and it stops once E_t <= eps~ (or E_t <= eps with ``stop_raw_eps``).

    ``forced_hat`` replays a given sequence of argmin decisions, and
    ``forced_blocks`` a sequence of (k, k2) block choices of the greedy rule
    (used when a run in another precision took a near-tie the other way)."""
    C = np.asarray(C, dtype=np.float64)
    n, m = C.shape
    cm = float(C.max()) if cmax is None else cmax
    st = approx_setup(r, c, s, eps, cm, gamma, smooth)
    g, rt, ct, L = st.gamma, st.r_t, st.c_t, st.L
    thr = eps if stop_raw_eps else st.eps_stop
    z_tilde = Dual.zeros(n, m) if z0 is None else z0.copy()
    z_check = z_tilde.copy()
    theta = 1.0
    trace = AspotTrace() if record else None
    phi_check = phi(C, g, rt, ct, s, z_check)
    z = z_check
    E = float("inf")
    t = 0
    converged = False
    while t < max_iter:
        z_bar = z_check.axpby(1.0 - theta, z_tilde, theta)
        grad = grad_phi(C, g, rt, ct, s, z_bar)
        z_new = z_bar.axpby(1.0, grad, -1.0 / (L * theta))
        z_grave = z_bar.axpby(1.0, z_new.axpby(1.0, z_tilde, -1.0), theta)
        z_tilde = z_new
        k = _choose_block(block_rule, t, C, g, rt, ct, s, z_grave)
        if forced_blocks is not None and t < len(forced_blocks):
            k = int(forced_blocks[t][0])
        z_hat = greenkhorn_step(C, g, rt, ct, s, z_grave, k)
        phi_hat = phi(C, g, rt, ct, s, z_hat)
        if forced_hat is not None and t < len(forced_hat):
            take = bool(forced_hat[t])
        else:
            take = phi_hat < phi_check
        z = z_hat if take else z_check
        phi_z = phi_hat if take else phi_check
        E = feas_error(C, g, rt, ct, s, z)
        k2 = k if block_rule == "cyclic" else _choose_block(block_rule, t, C, g, rt, ct, s, z)
        if forced_blocks is not None and t < len(forced_blocks):
            k2 = int(forced_blocks[t][1])
        z_check = greenkhorn_step(C, g, rt, ct, s, z, k2)
        phi_check = phi(C, g, rt, ct, s, z_check)
        if record:
            trace.k.append(k)
            trace.k2.append(k2)
            if block_rule == "greedy":
                trace.dec.append((block_decreases(C, g, rt, ct, s, z_grave), block_decreases(C, g, rt, ct, s, z)))
            trace.took_hat.append(take)
            trace.E.append(E)
            trace.theta.append(theta)
            trace.phi_grave.append(phi(C, g, rt, ct, s, z_grave))
            trace.phi_hat.append(phi_hat)
            trace.phi_z.append(phi_z)
            trace.phi_check_next.append(phi_check)
            trace.z_tilde.append(z_tilde.flat())
        theta = theta_next(theta)
        t += 1
        if not no_stop and E <= thr:
            converged = True
            break
    return SolveResult(z, t, E, st, converged, trace, z_check)


# --------------------------------------------------------------------------
# Feasible Sinkhorn baseline (extended OT with dummy nodes, Algorithm 3)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class SinkhornResult:
    u: np.ndarray        # extended potentials, length n+1 (or n when dropped)
    v: np.ndarray
    iters: int
    residual: float
    gamma: float
    eps_stop: float
    A: float
    r_ext: np.ndarray
    c_ext: np.ndarray
    converged: bool
    has_dummy_row: bool
    has_dummy_col: bool


def extended_cost(C, A) -> np.ndarray:
    """C~ = [[C, 0], [0^T, A]] (appendix, reduction to extended OT)."""
    n, m = C.shape
    Ce = np.zeros((n + 1, m + 1))
    Ce[:n, :m] = C
    Ce[n, m] = A
    return Ce


def tuned_gamma(r, c, eps, p) -> tuple:
    """Theorem 2 / Algorithm 3: H_min = min(H(r), H(c)),
    gamma = (2 eps / (49 H_min))^(1/p), eps' = H_min gamma^p."""
    hmin = min(entropy(r), entropy(c))
    gamma = (2.0 * eps / (49.0 * hmin)) ** (1.0 / p)
    return gamma, hmin * gamma ** p


def sinkhorn_pot(C, r, c, s, eps, gamma: Optional[float] = None, max_iter: int = 100000,
                 p_tune: float = 0.0, smooth: bool = True, cmax: Optional[float] = None,
                 no_stop: bool = False) -> SinkhornResult:
    """Feasible Sinkhorn for POT: alternate exact row and column scalings of
    the extended kernel exp(-C~/gamma) in the log domain,
      u <- u + log r_ext - log(B 1),   v <- v + log c_ext - log(B^T 1),
    until |B 1 - r_ext|_1 + |B^T 1 - c_ext|_1 <= eps'.  gamma, eps' and the
    smoothing come from Algorithm 2's setup (Section 4.1); with p_tune >= 1
    they come from the tuned rule of Theorem 2 instead."""
    C = np.asarray(C, dtype=np.float64)
    n, m = C.shape
    cm = float(C.max()) if cmax is None else cmax
    st = approx_setup(r, c, s, eps, cm, gamma, smooth)
    g, thr = st.gamma, st.eps_stop
    if p_tune >= 1.0:
        g, thr = tuned_gamma(r, c, eps, p_tune)
    A = 8.0 * cm / eps
    rt, ct = st.r_t, st.c_t
    dr, dc = ct.sum() - s, rt.sum() - s
    has_r, has_c = dr > 0, dc > 0
    r_ext = np.concatenate([rt, [dr]]) if has_r else rt.copy()
    c_ext = np.concatenate([ct, [dc]]) if has_c else ct.copy()
    Ce = extended_cost(C, A)[: n + (1 if has_r else 0), : m + (1 if has_c else 0)]
    Ke = -Ce / g
    u = np.zeros(Ce.shape[0])
    v = np.zeros(Ce.shape[1])
    res = float("inf")
    it = 0
    converged = False
    while it < max_iter:
        u = np.log(r_ext) - logsumexp(Ke + v[None, :], axis=1)
        v = np.log(c_ext) - logsumexp(Ke + u[:, None], axis=0)
        it += 1
        Lg = Ke + u[:, None] + v[None, :]
        res = float(np.abs(np.exp(logsumexp(Lg, axis=1)) - r_ext).sum()
                    + np.abs(np.exp(logsumexp(Lg, axis=0)) - c_ext).sum())
        if not no_stop and res <= thr:
            converged = True
            break
    return SinkhornResult(u, v, it, res, g, thr, A, r_ext, c_ext, converged, has_r, has_c)


def sinkhorn_plan_extended(C, res: SinkhornResult) -> np.ndarray:
    n, m = C.shape
    Ce = extended_cost(np.asarray(C, dtype=np.float64), res.A)
    Ce = Ce[: n + (1 if res.has_dummy_row else 0), : m + (1 if res.has_dummy_col else 0)]
    return np.exp(-Ce / res.gamma + res.u[:, None] + res.v[None, :])


# --------------------------------------------------------------------------
# Rounding and the objective
# --------------------------------------------------------------------------

def round_pot(Xt, r, c, s) -> np.ndarray:
    """ROUND-POT reading (R1-R4) of the rounding that Algorithm 2 cites.

    R1  a_i = min(1, r_i / (X~ 1)_i),        X' = diag(a) X~
    R2  b_j = min(1, c_j / (X'^T 1)_j),      X'' = X' diag(b)
    R3  m'' = 1^T X'' 1; if m'' >= s:        X = (s / m'') X''
    R4  else p = r - X'' 1, q = c - X''^T 1 (both >= 0),
        X = X'' + (s - m'') p q^T / (|p|_1 |q|_1)
    The result lies in U(r, c, s) whenever s <= min(|r|_1, |c|_1)."""
    Xt = np.asarray(Xt, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.minimum(1.0, r / Xt.sum(axis=1))
        a = np.where(np.isfinite(a), a, 1.0)
        X1 = a[:, None] * Xt
        b = np.minimum(1.0, c / X1.sum(axis=0))
        b = np.where(np.isfinite(b), b, 1.0)
    X2 = X1 * b[None, :]
    m2 = X2.sum()
    if m2 >= s:
        return (s / m2) * X2
    # p, q >= 0 by construction (R1, R2); the clamp only removes FP64 rounding
    p = np.maximum(r - X2.sum(axis=1), 0.0)
    q = np.maximum(c - X2.sum(axis=0), 0.0)
    return X2 + (s - m2) * np.outer(p, q) / (p.sum() * q.sum())


def altschuler_round(X, r, c) -> np.ndarray:
    """Rounding onto the balanced polytope U(r, c) (the Round routine that
    Algorithm 3 calls): scale rows down, scale columns down, then add the
    rank-one correction err_r err_c^T / |err_r|_1."""
    X = np.asarray(X, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        x = np.minimum(1.0, r / X.sum(axis=1))
        x = np.where(np.isfinite(x), x, 1.0)
        X = x[:, None] * X
        y = np.minimum(1.0, c / X.sum(axis=0))
        y = np.where(np.isfinite(y), y, 1.0)
        X = X * y[None, :]
    er = r - X.sum(axis=1)
    ec = c - X.sum(axis=0)
    if er.sum() > 0:
        X = X + np.outer(er, ec) / er.sum()
    return X


def objective(C, X) -> float:
    """<C, X> (Definition 1)."""
    return float((np.asarray(C, dtype=np.float64) * X).sum())


def primal_plan(C, gamma, z: Dual) -> np.ndarray:
    """Form primal: X~ = B(z) (Algorithm 2, after the loop)."""
    return np.exp(log_gibbs(C, gamma, z.u, z.v, z.w))


def entropic_primal(C, gamma, X, p, q) -> float:
    """Primal of the dual in Eq. (dual) divided by gamma, written from the
    slack LP form of the appendix (x = (vec X, p, q), d = (vec C, 0)):
        <C, X>/gamma + sum x (log x - 1) over all entries of X, p and q.
    For any x with X 1 + p = r, X^T 1 + q = c, 1^T X 1 = s and any z, weak
    duality gives entropic_primal(x) >= -phi(z)."""
    def xlogx(a):
        a = np.asarray(a, dtype=np.float64)
        out = np.zeros_like(a)
        pos = a > 0
        out[pos] = a[pos] * (np.log(a[pos]) - 1.0)
        return out.sum()
    return float((np.asarray(C) * X).sum() / gamma + xlogx(X) + xlogx(p) + xlogx(q))


def balanced_sinkhorn(C, a, b, gamma, iters: int = 20000, tol: float = 1e-13):
    """Textbook log-domain Sinkhorn for balanced entropic OT (|a|_1 = |b|_1),
    used only for the balanced-reduction check."""
    C = np.asarray(C, dtype=np.float64)
    K = -C / gamma
    f = np.zeros(C.shape[0])
    g = np.zeros(C.shape[1])
    for _ in range(iters):
        f = np.log(a) - logsumexp(K + g[None, :], axis=1)
        g = np.log(b) - logsumexp(K + f[:, None], axis=0)
        P = np.exp(K + f[:, None] + g[None, :])
        if np.abs(P.sum(axis=1) - a).sum() < tol:
            break
    return np.exp(K + f[:, None] + g[None, :])


# --------------------------------------------------------------------------
# Whole solves (primal, rounding, objective)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class PlanResult:
    X: np.ndarray
    objective: float
    iters: int
    E: float
    gamma: float
    converged: bool
    solve: object


def solve_aspot(C, r, c, s, eps, gamma=None, **kw) -> PlanResult:
    """Algorithm 2 end to end: loop, primal X~ = B(z^t), ROUND-POT, <C, X>."""
    C = np.asarray(C, dtype=np.float64)
    res = aspot(C, r, c, s, eps, gamma, **kw)
    Xt = primal_plan(C, res.setup.gamma, res.z)
    X = round_pot(Xt, r, c, s)
    return PlanResult(X, objective(C, X), res.iters, res.E, res.setup.gamma, res.converged, res)


def solve_sinkhorn(C, r, c, s, eps, gamma=None, literal_round: bool = False, **kw) -> PlanResult:
    """Feasible Sinkhorn end to end.  By default the top-left block of the
    extended plan is rounded with ROUND-POT against the original r, c, s;
    ``literal_round`` applies the balanced Round onto U(r_ext, c_ext) first and
    crops, as Algorithm 3 prints it (its block mass is s + X_{n+1,m+1})."""
    C = np.asarray(C, dtype=np.float64)
    n, m = C.shape
    res = sinkhorn_pot(C, r, c, s, eps, gamma, **kw)
    Xe = sinkhorn_plan_extended(C, res)
    if literal_round:
        X = altschuler_round(Xe, res.r_ext, res.c_ext)[:n, :m]
    else:
        X = round_pot(Xe[:n, :m], r, c, s)
    return PlanResult(X, objective(C, X), res.iters, res.residual, res.gamma, res.converged, res)
