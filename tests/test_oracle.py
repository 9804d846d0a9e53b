"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check is independent of the oracle's own formulas: finite differences,
second-order (Newton) minimisation, exact LPs, brute force, closed forms and
invariants stated in arXiv 2601.17196.  All problems are non-square (n != m)
with unequal masses so that a transposed operand or a swapped marginal fails.
"""
import math

import numpy as np
import pytest

import pot_workloads as W
from oracle import lp
from oracle import pot as O


def _tiny(seed=0, n=5, m=6, **kw):
    p = W.tiny(seed, n=n, m=m, **kw)
    return p, p.C.astype(np.float64)


def _newton_dual_opt(C, gamma, r, c, s, iters=60):
    """Minimise phi by Newton's method with the analytic Hessian (blocks
    diag(r(B)+e^u), B, r(B); diag(c(B)+e^v), c(B); |B|_1).  Independent of the
    first-order algorithms under test."""
    n, m = C.shape
    x = np.zeros(n + m + 1)
    for _ in range(iters):
        u, v, w = x[:n], x[n:n + m], x[-1]
        B = np.exp(-C / gamma + u[:, None] + v[None, :] + w)
        rB, cB, tot = B.sum(1), B.sum(0), B.sum()
        g = np.concatenate([rB + np.exp(u) - r, cB + np.exp(v) - c, [tot - s]])
        H = np.zeros((n + m + 1, n + m + 1))
        H[:n, :n] = np.diag(rB + np.exp(u))
        H[n:n + m, n:n + m] = np.diag(cB + np.exp(v))
        H[:n, n:n + m] = B
        H[n:n + m, :n] = B.T
        H[:n, -1] = H[-1, :n] = rB
        H[n:n + m, -1] = H[-1, n:n + m] = cB
        H[-1, -1] = tot
        step = np.linalg.solve(H, g)
        # damped Newton on a convex function: halve until phi decreases
        def phi_x(y):
            uu, vv, ww = y[:n], y[n:n + m], y[-1]
            return (np.exp(-C / gamma + uu[:, None] + vv[None, :] + ww).sum() + np.exp(uu).sum()
                    + np.exp(vv).sum() - uu @ r - vv @ c - ww * s)
        t = 1.0
        f0 = phi_x(x)
        while phi_x(x - t * step) > f0 and t > 1e-12:
            t *= 0.5
        x = x - t * step
        if np.abs(g).max() < 1e-15:
            break
    return O.Dual(x[:n], x[n:n + m], x[-1])


# ----------------------------------------------------------------- setup ---

def test_setup_closed_forms_small_dense():
    """Algorithm 2 setup on the 256-point workload: max C = 1, eps = 1e-3,
    |r| = 1 (no guard), |c| = 1.2 (guard 8*0.4/0.2 = 16, inactive)."""
    p = W.small_dense(0)
    st = O.approx_setup(p.r, p.c, p.s, p.eps, float(p.C.max()), p.gamma)
    assert float(p.C.max()) == 1.0
    assert st.eps_stop == pytest.approx(1.25e-4, rel=1e-15)
    assert st.eps_smooth == pytest.approx(1.25e-4, rel=1e-15)
    assert st.r_t.sum() == pytest.approx(1.0, rel=1e-14)            # (1-e/8)*1 + e/8
    assert st.c_t.sum() == pytest.approx((1 - 1.25e-4 / 8) * 1.2 + 1.25e-4 / 8, rel=1e-14)
    assert st.L == pytest.approx(3 * (st.r_t.sum() + st.c_t.sum() - 0.8) / 0.05, rel=1e-14)
    g = O.approx_setup(p.r, p.c, p.s, p.eps, 1.0, None).gamma
    assert g == pytest.approx(1e-3 / (4 * math.log(256)), rel=1e-15)


def test_setup_mass_guard_makes_budget_reachable():
    """With |r| = 1.5, s = 1.49, eps = 2: eps~ = 0.25, guard 8*0.01/0.5 = 0.16
    is active and gives |r~|_1 = 0.98*1.5 + 0.02 = 1.49 = s exactly."""
    r = np.full(10, 0.15)
    c = np.full(12, 1.6 / 12)
    st = O.approx_setup(r, c, 1.49, 2.0, 1.0, 0.1)
    assert st.eps_stop == pytest.approx(0.25)
    assert st.eps_smooth == pytest.approx(0.16)
    assert st.r_t.sum() == pytest.approx(1.49, rel=1e-14)
    assert st.c_t.sum() >= 1.49


def test_theta_schedule_identities():
    """theta_{t+1}/theta_t = sqrt(1 - theta_{t+1}) and theta_t <= 2/(t+2)
    (proof of Lemma 2, and the cited bound)."""
    th = 1.0
    for t in range(20000):
        nx = O.theta_next(th)
        assert nx / th == pytest.approx(math.sqrt(1.0 - nx), rel=1e-12)
        assert th <= 2.0 / (t + 2) * (1 + 1e-12)
        th = nx


def test_tuned_gamma_closed_form():
    """Theorem 2: gamma = (2 eps/(49 H_min))^(1/p) and eps' = H_min gamma^p,
    hence eps' = 2 eps / 49 for every p; H of a uniform vector of mass 1 is
    log n."""
    n = 64
    r = np.full(n, 1.0 / n)
    c = np.full(80, 1.3 / 80)
    assert O.entropy(r) == pytest.approx(math.log(n), rel=1e-14)
    for p in (1.0, 2.0, 5.0):
        g, e1 = O.tuned_gamma(r, c, 0.01, p)
        assert e1 == pytest.approx(2 * 0.01 / 49, rel=1e-12)
        hmin = min(O.entropy(r), O.entropy(c))
        assert g == pytest.approx((2 * 0.01 / (49 * hmin)) ** (1 / p), rel=1e-14)


# ------------------------------------------------------- dual, gradient ---

def test_gradient_matches_finite_differences():
    p, C = _tiny(1, n=4, m=5)
    rng = np.random.default_rng(0)
    z = O.Dual(rng.normal(size=4), rng.normal(size=5), 0.3)
    g = O.grad_phi(C, 0.2, p.r, p.c, p.s, z).flat()
    x0 = z.flat()
    h = 1e-6
    fd = np.zeros_like(x0)
    for k in range(x0.size):
        xp, xm = x0.copy(), x0.copy()
        xp[k] += h
        xm[k] -= h
        fp = O.phi(C, 0.2, p.r, p.c, p.s, O.Dual(xp[:4], xp[4:9], xp[9]))
        fm = O.phi(C, 0.2, p.r, p.c, p.s, O.Dual(xm[:4], xm[4:9], xm[9]))
        fd[k] = (fp - fm) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_greenkhorn_step_is_exact_block_minimiser(k):
    """Algorithm 1: after the u step dphi/du = 0 (sum_j B_ij + e^{u_i} = r_i,
    proof of Theorem 3); after the v step likewise; after the w step
    |B|_1 = s.  The step is idempotent and its decrease equals the closed
    form sum rho(r_i, r_i(B)+e^{u_i}) / rho(s, |B|_1) of the same proof."""
    p, C = _tiny(2)
    rng = np.random.default_rng(k)
    z = O.Dual(rng.normal(size=5) - 2, rng.normal(size=6) - 2, 0.5)
    zk = O.greenkhorn_step(C, 0.1, p.r, p.c, p.s, z, k)
    g = O.grad_phi(C, 0.1, p.r, p.c, p.s, zk)
    part = [g.u, g.v, np.array([g.w])][k]
    assert np.abs(part).max() < 1e-13
    zkk = O.greenkhorn_step(C, 0.1, p.r, p.c, p.s, zk, k)
    np.testing.assert_allclose(zkk.flat(), zk.flat(), atol=1e-13)
    S = O.phi(C, 0.1, p.r, p.c, p.s, z) - O.phi(C, 0.1, p.r, p.c, p.s, zk)
    assert S == pytest.approx(O.block_decreases(C, 0.1, p.r, p.c, p.s, z)[k], rel=1e-9)
    # the other blocks are untouched
    for j in range(3):
        if j != k:
            a = [z.u, z.v, np.array([z.w])][j]
            b = [zk.u, zk.v, np.array([zk.w])][j]
            np.testing.assert_array_equal(a, b)


def test_phi_strong_duality_with_slack_lp_primal():
    """Eq. (dual) is the dual of the entropic slack LP of the appendix: at the
    minimiser z* (found by Newton's method) the primal point
    x* = (B(z*), e^{u*}, e^{v*}) is feasible and its entropic objective equals
    -phi(z*); any other dual point gives -phi(z) below it (weak duality)."""
    p, C = _tiny(4)
    gam = 0.08
    z = _newton_dual_opt(C, gam, p.r, p.c, p.s)
    B = O.primal_plan(C, gam, z)
    pp, qq = np.exp(z.u), np.exp(z.v)
    np.testing.assert_allclose(B.sum(1) + pp, p.r, atol=1e-13)
    np.testing.assert_allclose(B.sum(0) + qq, p.c, atol=1e-13)
    assert B.sum() == pytest.approx(p.s, abs=1e-13)
    P = O.entropic_primal(C, gam, B, pp, qq)
    assert P == pytest.approx(-O.phi(C, gam, p.r, p.c, p.s, z), abs=1e-10)
    rng = np.random.default_rng(1)
    for _ in range(20):
        zr = O.Dual(z.u + rng.normal(size=5), z.v + rng.normal(size=6), z.w + rng.normal())
        assert -O.phi(C, gam, p.r, p.c, p.s, zr) <= P + 1e-12


# ------------------------------------------------------------- ASPOT ---

def test_aspot_descent_chain_and_lemma2():
    """Proof of Lemma 1: phi(z_grave) >= phi(z^) >= phi(z^t) >= phi(z_check^{t+1})
    every iteration, phi(z_check^t) non-increasing (proof of Theorem 3), and
    Lemma 2 in its sharp form delta_t <= (L/2) theta_{t-1}^2 |z* - z~^0|^2."""
    p, C = _tiny(3)
    eps = 0.05
    res = O.aspot(C, p.r, p.c, p.s, eps, None, max_iter=400, record=True, no_stop=True)
    st = res.setup
    tr = res.trace
    tol = 1e-12
    for t in range(res.iters):
        assert tr.phi_grave[t] >= tr.phi_hat[t] - tol
        assert tr.phi_hat[t] >= tr.phi_z[t] - tol
        assert tr.phi_z[t] >= tr.phi_check_next[t] - tol
        if t:
            assert tr.phi_check_next[t] <= tr.phi_check_next[t - 1] + tol
    zs = _newton_dual_opt(C, st.gamma, st.r_t, st.c_t, p.s)
    fstar = O.phi(C, st.gamma, st.r_t, st.c_t, p.s, zs)
    R2 = float(zs.flat() @ zs.flat())
    for t in range(1, res.iters):
        delta = tr.phi_check_next[t - 1] - fstar
        assert delta <= st.L / 2 * tr.theta[t - 1] ** 2 * R2 + 1e-12
        assert delta >= -1e-12


def test_aspot_reaches_the_dual_minimiser():
    """Run long with a tight threshold; the iterate approaches the unique
    minimiser of phi (strictly convex thanks to the e^u, e^v terms)."""
    p, C = _tiny(5)
    res = O.aspot(C, p.r, p.c, p.s, 1e-2, 0.1, max_iter=200000, stop_raw_eps=True)
    st = res.setup
    res = O.aspot(C, p.r, p.c, p.s, 1e-9, 0.1, max_iter=200000, stop_raw_eps=True)
    zs = _newton_dual_opt(C, st.gamma, res.setup.r_t, res.setup.c_t, p.s)
    assert res.converged
    np.testing.assert_allclose(res.z.flat(), zs.flat(), atol=2e-6)


def test_greedy_rule_theorem3_decrease_bound():
    """Proof of Theorem 3: with the greedy block choice the decrease
    S = phi(z^t) - phi(z_check^{t+1}) is at least E_t^2 / 63."""
    p, C = _tiny(3)
    res = O.aspot(C, p.r, p.c, p.s, 0.05, None, max_iter=300, record=True, block_rule="greedy",
                  no_stop=True)
    tr = res.trace
    for t in range(res.iters):
        S = tr.phi_z[t] - tr.phi_check_next[t]
        assert S >= tr.E[t] ** 2 / 63 * (1 - 1e-9) - 1e-14   # phi is O(1): FP64 rounding


def test_dual_radius_bounds_the_optimum():
    """Eq. (R): |u*|, |v*| <= R for the minimiser of phi."""
    p, C = _tiny(6)
    gam = 0.05
    zs = _newton_dual_opt(C, gam, p.r, p.c, p.s)
    R = O.dual_radius(p.r, p.c, p.s, gam, float(C.max()))
    assert np.abs(zs.u).max() <= R and np.abs(zs.v).max() <= R


# ---------------------------------------------------- rounding, LP, eps ---

def test_round_pot_lands_in_feasible_set_both_branches():
    rng = np.random.default_rng(0)
    r = rng.uniform(0.5, 1.5, 7)
    r /= r.sum()
    c = rng.uniform(0.5, 1.5, 9)
    c *= 1.3 / c.sum()
    for scale, s in ((0.05, 0.8), (3.0, 0.8), (0.5, 0.999)):
        Xt = rng.uniform(0, 1, (7, 9)) * scale / 7
        X = O.round_pot(Xt, r, c, s)
        assert (X >= 0).all()
        assert (X.sum(1) <= r * (1 + 1e-12)).all()
        assert (X.sum(0) <= c * (1 + 1e-12)).all()
        assert X.sum() == pytest.approx(s, rel=1e-13)


def test_lp_matches_bruteforce_partial_matching():
    """Uniform capacities 1/N: the POT LP optimum is (1/N) times the cheapest
    matching with k = s N edges."""
    for seed in range(3):
        p = W.tiny(seed, n=5, m=6, uniform=False)
        C = p.C.astype(np.float64)
        r = np.full(5, 0.2)
        c = np.full(6, 0.2)
        assert lp.pot_lp(C, r, c, 0.6) == pytest.approx(lp.kmatching_bruteforce(C, 3) * 0.2, abs=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_eps_approximation_against_exact_lp(seed):
    """Definition 1 / Theorem 1: with gamma = eps/(4 log n) both solvers return
    X in U(r, c, s) with LP* <= <C, X> <= LP* + eps."""
    p, C = _tiny(seed)
    LP = lp.pot_lp(C, p.r, p.c, p.s)
    for eps in (0.1, 0.05):
        for res in (O.solve_aspot(C, p.r, p.c, p.s, eps, None, max_iter=100000),
                    O.solve_sinkhorn(C, p.r, p.c, p.s, eps, None, max_iter=100000)):
            X = res.X
            assert res.converged
            assert (X >= 0).all() and X.sum() == pytest.approx(p.s, rel=1e-12)
            assert (X.sum(1) <= p.r * (1 + 1e-12)).all() and (X.sum(0) <= p.c * (1 + 1e-12)).all()
            assert LP - 1e-12 <= res.objective <= LP + eps


def test_gap_to_lp_shrinks_as_gamma_falls():
    p, C = _tiny(7)
    LP = lp.pot_lp(C, p.r, p.c, p.s)
    gaps = []
    for gam in (0.1, 0.05, 0.02, 0.01):
        res = O.solve_aspot(C, p.r, p.c, p.s, 1e-4, gam, max_iter=200000, stop_raw_eps=True)
        gaps.append(res.objective - LP)
    assert all(g >= -1e-12 for g in gaps)
    assert gaps[-1] < gaps[0] and gaps[-1] <= min(gaps[:-1]) * 1.05


def test_balanced_case_reduces_to_ot():
    """s = |r|_1 = |c|_1 = 1: the rounded plan is a balanced transport plan
    (X 1 = r, X^T 1 = c), its cost is within eps of the OT LP, and within eps
    of textbook balanced Sinkhorn at the same gamma."""
    p = W.tiny(8, n=6, m=7, mass_r=1.0, mass_c=1.0, s=1.0)
    C = p.C.astype(np.float64)
    eps, gam = 0.02, 0.02
    LP = lp.pot_lp(C, p.r, p.c, 1.0)
    res = O.solve_aspot(C, p.r, p.c, 1.0, eps, gam, max_iter=200000)
    np.testing.assert_allclose(res.X.sum(1), p.r, atol=1e-12)
    np.testing.assert_allclose(res.X.sum(0), p.c, atol=1e-12)
    assert LP - 1e-12 <= res.objective <= LP + eps
    Pb = O.balanced_sinkhorn(C, p.r, p.c, gam)
    assert abs(res.objective - O.objective(C, Pb)) <= eps
    rs = O.solve_sinkhorn(C, p.r, p.c, 1.0, eps, gam, max_iter=200000)
    assert not rs.solve.has_dummy_row and not rs.solve.has_dummy_col
    assert LP - 1e-12 <= rs.objective <= LP + eps


def test_literal_round_then_crop_overshoots_budget():
    """Appendix (extended OT): rounding onto U(r_ext, c_ext) and cropping
    gives a block of mass s + X_{n+1,m+1}, i.e. the infeasibility that the
    feasible formulation fixes; ROUND-POT of the block gives mass s.  A small
    dummy cost (eps = 4 gives A = 8 max C / eps = 2) and gamma = 0.5 make the
    corner entry visible in FP64 (at the experiments' settings it is about
    e^{-3000})."""
    p, C = _tiny(9)
    eps, gam = 4.0, 0.5
    rs = O.sinkhorn_pot(C, p.r, p.c, p.s, eps, gam, max_iter=100000)
    assert rs.A == pytest.approx(2.0)
    Xe = O.sinkhorn_plan_extended(C, rs)
    Xr = O.altschuler_round(Xe, rs.r_ext, rs.c_ext)
    corner = Xr[5, 6]
    assert corner > 1e-4
    assert Xr[:5, :6].sum() == pytest.approx(p.s + corner, rel=1e-12)
    lit = O.solve_sinkhorn(C, p.r, p.c, p.s, eps, gam, literal_round=True, max_iter=100000)
    fea = O.solve_sinkhorn(C, p.r, p.c, p.s, eps, gam, max_iter=100000)
    assert lit.X.sum() > p.s + 1e-4
    assert fea.X.sum() == pytest.approx(p.s, rel=1e-13)


def test_sqeuclid_cost_definition():
    """Plain distances on integer points, where every value is exact."""
    X = np.array([[0.0, 0.0], [1.0, 2.0], [3.0, 1.0]])
    Y = np.array([[1.0, 1.0], [0.0, 3.0]])
    C = O.sqeuclid_cost(X, Y, 1.0)
    np.testing.assert_array_equal(C, [[2, 9], [1, 2], [4, 13]])
    np.testing.assert_array_equal(O.sqeuclid_cost(X, Y), np.array([[2, 9], [1, 2], [4, 13]]) / 13)


def test_feasibility_error_is_l1_norm_of_gradient():
    """With p = e^u and q = e^v, E(t) of Section 3.1 is exactly |grad phi|_1
    (the gradient itself is pinned by finite differences above)."""
    p, C = _tiny(10)
    rng = np.random.default_rng(3)
    for _ in range(5):
        z = O.Dual(rng.normal(size=5) - 2, rng.normal(size=6) - 2, rng.normal())
        E = O.feas_error(C, 0.07, p.r, p.c, p.s, z)
        assert E == pytest.approx(np.abs(O.grad_phi(C, 0.07, p.r, p.c, p.s, z).flat()).sum(), rel=1e-13)


def test_greedy_trace_and_replay():
    """The greedy rule's recorded blocks are the argmax of the recorded exact
    decreases (ties to the lower index); replaying a run's own decisions
    reproduces it exactly, and forcing other blocks is obeyed.  (The GPU
    parity tests replay the GPU's decisions through this option.)"""
    p = W.small_dense(6, n=40, m=52)
    C = p.C.astype(np.float64)
    free = O.aspot(C, p.r, p.c, p.s, 0.05, None, max_iter=30, no_stop=True, block_rule="greedy", record=True)
    for t in range(30):
        d_grave, d_z = (np.asarray(x) for x in free.trace.dec[t])
        assert free.trace.k[t] == int(np.argmax(d_grave))
        assert free.trace.k2[t] == int(np.argmax(d_z))
    rep = O.aspot(C, p.r, p.c, p.s, 0.05, None, max_iter=30, no_stop=True, block_rule="greedy", record=True,
                  forced_hat=free.trace.took_hat, forced_blocks=list(zip(free.trace.k, free.trace.k2)))
    np.testing.assert_array_equal(rep.z.u, free.z.u)
    np.testing.assert_array_equal(rep.z.v, free.z.v)
    forced = [(0, 1)] * 30
    other = O.aspot(C, p.r, p.c, p.s, 0.05, None, max_iter=30, no_stop=True, block_rule="greedy", record=True,
                    forced_blocks=forced)
    assert other.trace.k == [0] * 30 and other.trace.k2 == [1] * 30
    assert np.abs(other.z.u - free.z.u).max() > 1e-6
