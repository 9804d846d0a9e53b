"""GPU parity on degenerate inputs, against the FP64 oracle: the balanced
case (s equal to both masses) and s equal to the smaller mass, where
ASPOT's slacks only decay slowly (reading N17) and the rounding must give
exact marginals; a deep partial problem (s much smaller than the masses);
a single row, a single column and a 1 x 1 problem; points of zero mass.

ASPOT is compared with the oracle replaying the GPU's argmin decisions (a
near-tie of phi(z^) and phi(z_check) may go the other way in FP32), after a
fixed number of iterations where it does not converge, else at the GPU's
own stop; Sinkhorn at its converged stop.  Tolerances as in the other
parity tests: potentials 2e-5 (1 + |u|), objectives 1e-5 relative, rounded
plans feasible in FP64 to 1e-6."""
import numpy as np
import pytest
import torch

import paper_2601_17196_gb300 as pkg
import pot_workloads as W
from oracle import pot as O

pytestmark = pytest.mark.gpu


def _t(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _dense(C, r, c, s):
    Ct = torch.tensor(np.ascontiguousarray(C, dtype=np.float32), device="cuda")
    return pkg.DeviceProblem(pkg.COST_DENSE_F32, _t(r), _t(c), s, C=Ct, cost_scale=1.0)


def _plan(C, res):
    f, g, p, q = (_np(x) for x in (res.plan.f, res.plan.g, res.plan.p, res.plan.q))
    return np.exp(f[:, None] + g[None, :] - res.cost_scale * C / res.gamma) + float(res.plan.kappa.item()) * np.outer(p, q)


def _feasible(X, r, c, s, tol=1e-6):
    assert (X >= 0).all()
    assert (X.sum(1) <= r * (1 + tol) + 1e-15).all()
    assert (X.sum(0) <= c * (1 + tol) + 1e-15).all()
    assert abs(X.sum() - s) <= tol * s


def _aspot_vs_oracle(C, r, c, s, eps, gamma, fixed=None, tol=1e-6):
    dp = _dense(C, r, c, s)
    if fixed:
        res = pkg.aspot_solve(dp, gamma, eps, max_iter=fixed, flags=pkg.FLAG_NO_STOP | pkg.FLAG_TRACE, check_every=9)
        assert res.iters == fixed
    else:
        res = pkg.aspot_solve(dp, gamma, eps, max_iter=20000, flags=pkg.FLAG_TRACE)
        assert res.status == 0 and res.err_final <= res.eps_stop
    took = res.trace[:, 3] > 0.5
    ora = O.solve_aspot(C, r, c, s, eps, gamma, max_iter=res.iters, no_stop=True, forced_hat=list(took),
                        cmax=float(C.max()))
    z = ora.solve.z
    np.testing.assert_allclose(_np(res.plan.u), z.u, rtol=0, atol=2e-5 * (1 + np.abs(z.u).max()))
    np.testing.assert_allclose(_np(res.plan.v), z.v, rtol=0, atol=2e-5 * (1 + np.abs(z.v).max()))
    assert abs(res.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    X = _plan(C, res)
    _feasible(X, r, c, s, tol)
    return res, X


def _sinkhorn_vs_oracle(C, r, c, s, eps, gamma, tol=1e-6):
    res = pkg.sinkhorn_pot_solve(_dense(C, r, c, s), gamma, eps, max_iter=20000)
    ora = O.solve_sinkhorn(C, r, c, s, eps, gamma, max_iter=20000)
    assert res.status == 0 and abs(res.iters - ora.iters) <= 1
    assert abs(res.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    X = _plan(C, res)
    _feasible(X, r, c, s, tol)
    return res, X


def _cost(seed, n, m):
    pb = W.small_dense(seed, n=n, m=m)
    return pb, pb.C.astype(np.float64)


@pytest.mark.parametrize("mass_c", [1.0, 1.3])
def test_s_equal_to_a_full_mass(mass_c):
    """s = |r|_1 = 1 (balanced when |c|_1 = 1 too): every row must be fully
    transported, so the rounded plan has X 1 = r.  The rank-one fill of the
    rounding then makes each row tight, X 1 = X''1 + p with p = r - X''1
    formed from an FP32 pass, so the plan re-evaluated in FP64 meets r up to
    that pass's relative error (<= 5e-6 in e^lse): the marginals are checked
    to 1e-5 here instead of 1e-6."""
    pb, C = _cost(21, 120, 140)
    n, m = C.shape
    r, c = np.full(n, 1.0 / n), np.full(m, mass_c / m)
    _, X = _aspot_vs_oracle(C, r, c, 1.0, 1e-3, 0.05, fixed=150, tol=1e-5)
    assert np.abs(X.sum(1) - r).sum() <= 1e-5
    if mass_c == 1.0:
        assert np.abs(X.sum(0) - c).sum() <= 1e-5
    _, Xs = _sinkhorn_vs_oracle(C, r, c, 1.0, 1e-3, 0.05, tol=1e-5)
    assert np.abs(Xs.sum(1) - r).sum() <= 1e-5


def test_deep_partial_transport():
    """s = 0.05 against masses 1.0 and 1.3."""
    pb, C = _cost(22, 150, 170)
    _aspot_vs_oracle(C, pb.r, pb.c, 0.05, 1e-3, 0.05)
    _sinkhorn_vs_oracle(C, pb.r, pb.c, 0.05, 1e-3, 0.05)


@pytest.mark.parametrize("n,m", [(1, 37), (41, 1), (1, 1)])
def test_single_row_or_column(n, m):
    rng = np.random.default_rng(n * 100 + m)
    C = rng.random((n, m))
    C = C / C.max()
    r, c = np.full(n, 1.0 / n), np.full(m, 1.2 / m)
    _aspot_vs_oracle(C, r, c, 0.8, 1e-3, 0.05)
    _sinkhorn_vs_oracle(C, r, c, 0.8, 1e-3, 0.05)


def test_points_of_zero_mass():
    """Every 7th row and 5th column carry no mass: the smoothing of
    Algorithm 2's setup makes their smoothed masses positive, and the
    rounding (against the original r, c) leaves them empty."""
    pb, C = _cost(23, 120, 140)
    r, c = pb.r.copy(), pb.c.copy()
    r[::7] = 0.0
    c[::5] = 0.0
    r *= pb.r.sum() / r.sum()
    c *= pb.c.sum() / c.sum()
    _, X = _aspot_vs_oracle(C, r, c, pb.s, 1e-3, 0.05)
    assert X[::7].max() == 0.0 and X[:, ::5].max() == 0.0
    _, Xs = _sinkhorn_vs_oracle(C, r, c, pb.s, 1e-3, 0.05)
    assert Xs[::7].max() == 0.0 and Xs[:, ::5].max() == 0.0
