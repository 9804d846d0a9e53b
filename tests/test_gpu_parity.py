"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Tolerances (FP32 passes, FP64 potentials and bookkeeping):
  * per-pass log-sums: |lse_gpu - lse_fp64| <= 5e-6 + 2e-7 |lse| (relative
    error of the sums; each logit is rounded once in FP32 after the exact
    hi/lo potential add, so its error is relative to its own magnitude; then
    ex2.approx and FP32 partial sums).
  * fixed-iteration ASPOT: potentials within 2e-5 (1 + |u|) after 60
    iterations, with the oracle replaying the GPU's argmin decisions.
  * converged solves: |objective difference| <= 1e-5 relative, final E_t below
    the threshold, and the GPU plan feasible in FP64 to 1e-6.
"""
import numpy as np
import pytest
import torch

import paper_2601_17196_gb300 as pkg
import pot_workloads as W
from oracle import pot as O

pytestmark = pytest.mark.gpu


def _dev(pb, **kw):
    return pkg.DeviceProblem.from_workload(pb, device="cuda", **kw)


def _t(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _plan_fp64(C, plan, gamma, cost_scale):
    f, g, p, q = _np(plan.f), _np(plan.g), _np(plan.p), _np(plan.q)
    kap = float(plan.kappa.item())
    return np.exp(f[:, None] + g[None, :] - cost_scale * C / gamma) + kap * np.outer(p, q)


def _check_feasible(X, r, c, s, tol=1e-6):
    assert (X >= 0).all()
    assert (X.sum(1) <= r * (1 + tol) + 1e-15).all()
    assert (X.sum(0) <= c * (1 + tol) + 1e-15).all()
    assert abs(X.sum() - s) <= tol * s


# ------------------------------------------------------------ one pass ---

@pytest.mark.parametrize("n,m", [(300, 457), (1, 1), (7, 300), (513, 129)])
def test_marginals_dense(n, m):
    pb = W.small_dense(1, n=n, m=m)
    C = pb.C.astype(np.float64)
    rng = np.random.default_rng(n + m)
    gam = 0.02
    for lo, hi in ((-5.0, 5.0), (-400.0, 300.0)):
        u, v, w = rng.uniform(lo, hi, n), rng.uniform(lo, hi, m), float(rng.uniform(lo, hi))
        dp = _dev(pb)
        lr, lc, tot = pkg.pot_marginals(dp, gam, _t(u), _t(v), w)
        L = O.log_gibbs(C, gam, u, v, w)
        er, ec = O.logsumexp(L, axis=1), O.logsumexp(L, axis=0)
        assert np.all(np.abs(_np(lr) - er) <= 5e-6 + 2e-7 * np.abs(er))
        assert np.all(np.abs(_np(lc) - ec) <= 5e-6 + 2e-7 * np.abs(ec))
        ltot = O.logsumexp(L)
        if -700 < ltot < 700:
            assert abs(np.log(tot) - ltot) <= 5e-6 + 2e-7 * abs(ltot)


@pytest.mark.parametrize("kind,d", [(pkg.COST_SQEUCLID_F32, 3), (pkg.COST_SQEUCLID_F32, 2),
                                    (pkg.COST_SQEUCLID_BF16, 128), (pkg.COST_SQEUCLID_BF16, 64),
                                    # CUDA-core paths: small d in registers, and the generic loop over d
                                    (pkg.COST_SQEUCLID_F32, 7), (pkg.COST_SQEUCLID_F16, 3),
                                    (pkg.COST_SQEUCLID_F16, 33), (pkg.COST_SQEUCLID_BF16, 3),
                                    (pkg.COST_SQEUCLID_BF16, 20)])
def test_marginals_sqeuclid(kind, d):
    n, m = 385, 521
    if kind == pkg.COST_SQEUCLID_BF16 and d % 64 == 0:
        pb = W.cloud_32k(2, n=n, m=m, d=d)
    else:
        rng = np.random.default_rng(d)
        X, Y = rng.uniform(0, 1, (n, d)), rng.uniform(0, 1, (m, d))
        if kind == pkg.COST_SQEUCLID_F16:                  # the values the kernel sees
            X, Y = X.astype(np.float16).astype(np.float64), Y.astype(np.float16).astype(np.float64)
        elif kind == pkg.COST_SQEUCLID_BF16:
            Xb, Yb = W.to_bf16_bits(X), W.to_bf16_bits(Y)
            X, Y = W.from_bf16_bits(Xb), W.from_bf16_bits(Yb)
        else:
            X, Y = X.astype(np.float32).astype(np.float64), Y.astype(np.float32).astype(np.float64)
        pb = W.Problem("pts", np.full(n, 1.0 / n), np.full(m, 1.3 / m), 0.8, 0.05, 1e-3, X=X, Y=Y)
        if kind == pkg.COST_SQEUCLID_BF16:
            pb.X_bf16, pb.Y_bf16 = Xb, Yb
    Dm = O.sqeuclid_cost(pb.X, pb.Y, 1.0)
    scale = 1.0 / Dm.max()
    pb.cost_scale = scale
    C = Dm * scale
    dp = _dev(pb, kind=kind)
    rng = np.random.default_rng(7)
    gam = 0.02
    u, v, w = rng.uniform(-30, 5, n), rng.uniform(-30, 5, m), 3.0
    lr, lc, tot = pkg.pot_marginals(dp, gam, _t(u), _t(v), w)
    L = O.log_gibbs(C, gam, u, v, w)
    # The generic loop over d (d > 4, not a tensor-core size) forms the cost from
    # FP32 dot products and squared norms.  A d-term FP32 sum errs by at most
    # about d 2^-24 times the sum of magnitudes, so a cost entry by
    # 2 (d + 2) 2^-24 (|x|^2 + |y|^2), and a logit by that x scale / gamma.
    # The register path (d <= 4) and the tensor-core paths keep 2e-5.
    tol = 2e-5
    if d > 4 and not (kind == pkg.COST_SQEUCLID_BF16 and d % 64 == 0):
        mag = (pb.X ** 2).sum(1).max() + (pb.Y ** 2).sum(1).max()
        tol += 2 * (d + 2) * 2.0 ** -24 * mag * scale / gam
    np.testing.assert_allclose(_np(lr), O.logsumexp(L, axis=1), rtol=0, atol=tol)
    np.testing.assert_allclose(_np(lc), O.logsumexp(L, axis=0), rtol=0, atol=tol)
    assert pkg.pot_cost_max(dp) == pytest.approx(Dm.max(), rel=2e-6 * max(1, (d + 2) / 6))


# ----------------------------------------------------------- solvers ---

# the small solves run in the single-cluster loop unless FLAG_STAGED asks for
# the separate kernels: both loops are held to the same bars
LOOPS = [pytest.param(0, id="cluster"), pytest.param(pkg.FLAG_STAGED, id="staged")]


@pytest.mark.parametrize("loop", LOOPS)
def test_aspot_fixed_iterations_match_oracle(loop):
    pb = W.small_dense(3, n=200, m=233)
    C = pb.C.astype(np.float64)
    K = 60
    res = pkg.aspot_solve(_dev(pb), pb.gamma, pb.eps, max_iter=K, flags=pkg.FLAG_NO_STOP | pkg.FLAG_TRACE | loop,
                          check_every=9)
    assert res.iters == K and res.cluster_loop == (0 if loop else 1)
    took = res.trace[:, 3] > 0.5
    ora = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=K, no_stop=True, forced_hat=took,
                  record=True)
    free = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=K, no_stop=True, record=True)
    # decisions the FP64 run would take differently must be near-ties
    for t in range(K):
        if free.trace.took_hat[t] != took[t]:
            assert abs(free.trace.phi_hat[t] - free.trace.phi_check_next[max(t - 1, 0)]) < 1e-6
    u, v, w = _np(res.plan.u), _np(res.plan.v), float(res.plan.w.item())
    np.testing.assert_allclose(u, ora.z.u, rtol=0, atol=2e-5 * (1 + np.abs(ora.z.u).max()))
    np.testing.assert_allclose(v, ora.z.v, rtol=0, atol=2e-5 * (1 + np.abs(ora.z.v).max()))
    assert w == pytest.approx(ora.z.w, abs=2e-5 * (1 + abs(ora.z.w)))
    np.testing.assert_allclose(res.trace[:, 0], ora.trace.E, rtol=1e-3, atol=1e-7)


def _greedy_codes(trace):
    code = np.rint(trace[:, 3]).astype(np.int64)
    return (code & 1) > 0, (code >> 1) & 3, (code >> 3) & 3


def _near_tie(dec, k, mass=1.5, delta=1e-5):
    """The decrease of block k is within the GPU's error of the largest one.
    Each decrease D = sum rho(a, b), rho(a, b) = b - a + a log(a/b), is formed
    from FP32-pass sums b with relative error <= delta; to first order that
    moves D by delta sum|b - a| <= delta sqrt(2 D sum a) (Cauchy-Schwarz with
    rho(a, b) ~ (b - a)^2 / (2a)), which near convergence is of the size of D
    itself, so block choices there are near-ties."""
    dec = np.asarray(dec, dtype=np.float64)
    dmax = dec.max()
    err = delta * (np.sqrt(2 * max(dmax, 0.0) * mass) + np.sqrt(2 * max(dec[k], 0.0) * mass))
    return dmax - dec[k] <= 1e-12 + 2 * err


@pytest.mark.parametrize("loop", LOOPS)
def test_aspot_greedy_fixed_iterations_match_oracle(loop):
    """Greedy block rule (the choice in Theorem 3's proof): 60 iterations with
    the oracle replaying the GPU's argmin and block decisions; every decision
    the free FP64 run takes differently before the runs part is a near-tie."""
    pb = W.small_dense(3, n=200, m=233)
    C = pb.C.astype(np.float64)
    K = 60
    res = pkg.aspot_solve(_dev(pb), pb.gamma, pb.eps, max_iter=K, flags=pkg.FLAG_NO_STOP | pkg.FLAG_TRACE | loop,
                          check_every=9, block_rule=pkg.BLOCK_GREEDY)
    assert res.iters == K and res.cluster_loop == (0 if loop else 1)
    took, k, k2 = _greedy_codes(res.trace)
    assert set(k.tolist()) <= {0, 1, 2} and set(k2.tolist()) <= {0, 1, 2}
    assert len(set(k.tolist())) >= 2            # the rule is not a fixed block on this instance
    ora = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=K, no_stop=True, forced_hat=took,
                  forced_blocks=list(zip(k, k2)), block_rule="greedy", record=True)
    free = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=K, no_stop=True, block_rule="greedy",
                   record=True)
    assert _first_split_is_near_tie(free, took, k, k2)
    assert ora.trace.k == k.tolist() and ora.trace.k2 == k2.tolist()
    u, v, w = _np(res.plan.u), _np(res.plan.v), float(res.plan.w.item())
    np.testing.assert_allclose(u, ora.z.u, rtol=0, atol=2e-5 * (1 + np.abs(ora.z.u).max()))
    np.testing.assert_allclose(v, ora.z.v, rtol=0, atol=2e-5 * (1 + np.abs(ora.z.v).max()))
    assert w == pytest.approx(ora.z.w, abs=2e-5 * (1 + abs(ora.z.w)))
    np.testing.assert_allclose(res.trace[:, 0], ora.trace.E, rtol=1e-3, atol=1e-7)


def _first_split_is_near_tie(free, took, k, k2):
    """Up to the first iteration where the free FP64 greedy run decides
    differently from the GPU, the decisions agree; that one is a near-tie."""
    for t in range(min(len(took), len(free.trace.k))):
        if free.trace.k[t] != k[t]:
            return _near_tie(free.trace.dec[t][0], k[t])
        if free.trace.took_hat[t] != took[t]:
            return abs(free.trace.phi_hat[t] - free.trace.phi_check_next[max(t - 1, 0)]) < 1e-6
        if free.trace.k2[t] != k2[t]:
            return _near_tie(free.trace.dec[t][1], k2[t])
    return True


@pytest.mark.parametrize("loop", LOOPS)
def test_aspot_greedy_converged_matches_oracle(loop):
    """Greedy rule to the stop threshold on the 256-point workload.  The
    oracle replays the GPU's decisions for the GPU's iteration count: the
    objectives agree to 1e-5 relative, the oracle's E_t is below the
    threshold there too, the plan is feasible, and the free FP64 run parts
    from the GPU's decisions only at a near-tie."""
    pb = W.small_dense(0)
    C = pb.C.astype(np.float64)
    res = pkg.aspot_solve(_dev(pb), pb.gamma, pb.eps, max_iter=5000, flags=pkg.FLAG_TRACE | loop,
                          block_rule=pkg.BLOCK_GREEDY)
    assert res.status == 0 and res.cluster_loop == (0 if loop else 1)
    assert res.err_final <= res.eps_stop
    took, k, k2 = _greedy_codes(res.trace)
    ora = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=res.iters, no_stop=True,
                        block_rule="greedy", forced_hat=took, forced_blocks=list(zip(k, k2)))
    assert ora.E <= res.eps_stop * (1 + 1e-3)
    assert abs(res.err_final - ora.E) <= 1e-3 * ora.E
    assert abs(res.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    X = _plan_fp64(C, res.plan, res.gamma, res.cost_scale)
    _check_feasible(X, pb.r, pb.c, pb.s)
    free = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=res.iters, no_stop=True,
                   block_rule="greedy", record=True)
    assert _first_split_is_near_tie(free, took, k, k2)


@pytest.mark.parametrize("solver", ["aspot", "sinkhorn"])
def test_converged_small_dense(solver):
    """The 256-point workload (Section 4.1 stand-in) to the stop threshold."""
    pb = W.small_dense(0)
    C = pb.C.astype(np.float64)
    if solver == "aspot":
        res = pkg.aspot_solve(_dev(pb), pb.gamma, pb.eps, max_iter=5000)
        ora = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=5000)
    else:
        res = pkg.sinkhorn_pot_solve(_dev(pb), pb.gamma, pb.eps, max_iter=5000)
        ora = O.solve_sinkhorn(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=5000)
    assert res.status == 0
    assert res.err_final <= res.eps_stop
    assert abs(res.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    X = _plan_fp64(C, res.plan, res.gamma, res.cost_scale)
    _check_feasible(X, pb.r, pb.c, pb.s)
    assert O.objective(C, X) == pytest.approx(res.objective, rel=1e-6)
    # the returned duals reach the threshold in FP64 as well
    if solver == "aspot":
        st = O.approx_setup(pb.r, pb.c, pb.s, pb.eps, 1.0, pb.gamma)
        z = O.Dual(_np(res.plan.u), _np(res.plan.v), float(res.plan.w.item()))
        E = O.feas_error(C, pb.gamma, st.r_t, st.c_t, pb.s, z)
        assert E == pytest.approx(res.err_final, rel=1e-3, abs=1e-9)


def test_pot_round_matches_oracle_reading():
    pb = W.small_dense(4, n=150, m=170)
    C = pb.C.astype(np.float64)
    ora = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=40, no_stop=True)
    for shift in (0.0, 2.0, -3.0):          # move w to exercise both branches (R3 and R4)
        z = ora.z
        dp = _dev(pb)
        plan, branch = pkg.pot_round(dp, pb.gamma, _t(z.u), _t(z.v), z.w + shift)
        Xo = O.round_pot(O.primal_plan(C, pb.gamma, O.Dual(z.u, z.v, z.w + shift)), pb.r, pb.c, pb.s)
        X = _plan_fp64(C, plan, pb.gamma, 1.0)
        np.testing.assert_allclose(X, Xo, rtol=0, atol=1e-5 * Xo.max())
        _check_feasible(X, pb.r, pb.c, pb.s)
        Xd = _np(pkg.pot_plan_dense(dp, plan, pb.gamma)).astype(np.float64)
        np.testing.assert_allclose(Xd, X, rtol=1e-5, atol=1e-7 * X.max())
        m2 = (O.primal_plan(C, pb.gamma, O.Dual(z.u, z.v, z.w + shift))).sum()
        assert branch in (3, 4)
        obj = pkg.pot_objective(dp, plan, pb.gamma)
        assert obj == pytest.approx(O.objective(C, Xo), rel=1e-5)


def test_invalid_arguments_are_rejected():
    pb = W.small_dense(0, n=32, m=40)
    dp = _dev(pb)
    bad = pkg.DeviceProblem(dp.kind, dp.r, dp.c, 5.0, C=dp.C, cost_scale=1.0)   # s > min mass
    with pytest.raises(pkg.PotError) as e:
        pkg.aspot_solve(bad, 0.05, 1e-3)
    assert e.value.status == 1
    with pytest.raises(pkg.PotError) as e:
        pkg.aspot_solve(dp, 0.05, 1e-3, ws=torch.empty(1024, dtype=torch.uint8, device="cuda"))
    assert e.value.status in (1, 2)
    nanr = dp.r.clone()
    nanr[3] = float("nan")
    with pytest.raises(pkg.PotError):
        pkg.aspot_solve(pkg.DeviceProblem(dp.kind, nanr, dp.c, 0.5, C=dp.C, cost_scale=1.0), 0.05, 1e-3)


def test_max_iter_reports_noconv_with_feasible_plan():
    pb = W.small_dense(0)
    C = pb.C.astype(np.float64)
    res = pkg.aspot_solve(_dev(pb), pb.gamma, pb.eps, max_iter=5)
    assert res.status == 4 and res.iters == 5
    _check_feasible(_plan_fp64(C, res.plan, res.gamma, res.cost_scale), pb.r, pb.c, pb.s)


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("gamma", [0.1, 0.03, 0.01])
def test_dense_4096_full_size_properties(gamma, rule):
    """n = m = 4096, 64-D, FP32 cost, both block rules: the GPU solve is
    checked in FP64 at its own duals (E_t below the threshold, objective and
    feasibility of the rounded plan); the oracle's full solve at this size is
    too slow for a test."""
    pb = W.dense_4096(0, gamma=gamma)
    C = pb.C.astype(np.float64)
    res = pkg.aspot_solve(_dev(pb), pb.gamma, pb.eps, max_iter=20000, block_rule=rule)
    assert res.status == 0
    st = O.approx_setup(pb.r, pb.c, pb.s, pb.eps, 1.0, pb.gamma)
    z = O.Dual(_np(res.plan.u), _np(res.plan.v), float(res.plan.w.item()))
    E = O.feas_error(C, pb.gamma, st.r_t, st.c_t, pb.s, z)
    assert E <= res.eps_stop * 1.001
    X = _plan_fp64(C, res.plan, res.gamma, res.cost_scale)
    _check_feasible(X, pb.r, pb.c, pb.s)
    assert O.objective(C, X) == pytest.approx(res.objective, rel=1e-5)


@pytest.mark.parametrize("p_tune", [1.5, 2.0, 4.0])
def test_tuned_gamma_sinkhorn_matches_oracle(p_tune):
    """Theorem 2 / Algorithm 3: gamma = (2 eps / (49 H_min))^(1/p) and the
    stop threshold eps' = H_min gamma^p; same iterations and objective as the
    oracle's tuned Sinkhorn."""
    pb = W.small_dense(2, n=180, m=210)
    C = pb.C.astype(np.float64)
    eps = 0.05
    res = pkg.sinkhorn_pot_solve(_dev(pb), 0.0, eps, max_iter=20000, p_tune=p_tune)
    ora = O.solve_sinkhorn(C, pb.r, pb.c, pb.s, eps, None, max_iter=20000, p_tune=p_tune)
    g, e1 = O.tuned_gamma(pb.r, pb.c, eps, p_tune)
    assert res.gamma == pytest.approx(g, rel=1e-12)
    assert res.eps_stop == pytest.approx(e1, rel=1e-12)
    assert res.status == 0 and abs(res.iters - ora.iters) <= 1
    assert abs(res.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    _check_feasible(_plan_fp64(C, res.plan, res.gamma, res.cost_scale), pb.r, pb.c, pb.s)


@pytest.mark.parametrize("kind,d", [(pkg.COST_SQEUCLID_F32, 3), (pkg.COST_SQEUCLID_F16, 3),
                                    (pkg.COST_SQEUCLID_F32, 7), (pkg.COST_SQEUCLID_BF16, 20)])
def test_aspot_solve_on_point_clouds(kind, d):
    """ASPOT to its threshold on point clouds of each storage kind through the
    CUDA-core paths (registers for d <= 4, the generic loop otherwise), the
    oracle replaying the GPU's argmin decisions at the GPU's iteration count:
    objectives to 1e-5 relative, feasible rounded plan."""
    n, m = 210, 170
    rng = np.random.default_rng(100 + d)
    X, Y = rng.uniform(0, 1, (n, d)), rng.uniform(0, 1, (m, d)) * 0.8 + 0.1
    Xb = Yb = None
    if kind == pkg.COST_SQEUCLID_F16:
        X, Y = X.astype(np.float16).astype(np.float64), Y.astype(np.float16).astype(np.float64)
    elif kind == pkg.COST_SQEUCLID_BF16:
        Xb, Yb = W.to_bf16_bits(X), W.to_bf16_bits(Y)
        X, Y = W.from_bf16_bits(Xb), W.from_bf16_bits(Yb)
    else:
        X, Y = X.astype(np.float32).astype(np.float64), Y.astype(np.float32).astype(np.float64)
    r, c = np.full(n, 1.0 / n), np.full(m, 1.25 / m)
    pb = W.Problem("pts", r, c, 0.8, 0.05, 1e-3, X=X, Y=Y, X_bf16=Xb, Y_bf16=Yb)
    Dm = O.sqeuclid_cost(X, Y, 1.0)
    pb.cost_scale = 1.0 / Dm.max()
    C = Dm * pb.cost_scale
    res = pkg.aspot_solve(_dev(pb, kind=kind), pb.gamma, pb.eps, max_iter=5000, flags=pkg.FLAG_TRACE)
    assert res.status == 0 and res.err_final <= res.eps_stop
    took = res.trace[:, 3] > 0.5
    ora = O.solve_aspot(C, r, c, pb.s, pb.eps, pb.gamma, max_iter=res.iters, no_stop=True, forced_hat=list(took),
                        cmax=1.0)
    assert abs(res.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    _check_feasible(_plan_fp64(C, res.plan, res.gamma, 1.0), r, c, pb.s)


@pytest.mark.parametrize("rule", [0, 1])
def test_aspot_resume_continues_exactly(rule):
    """Checkpoint / resume: a solve stopped after 61 iterations (not a multiple
    of 3, so the cyclic rule must go on with block 61 mod 3), exported with
    aspot_state_export and resumed to 122 iterations, ends bit for bit where an
    uninterrupted 122-iteration solve ends."""
    pb = W.small_dense(3, n=200, m=233)
    dp = _dev(pb)
    flags = pkg.FLAG_NO_STOP
    ws = torch.empty(pkg.binding.workspace_bytes(dp, flags) + 256, dtype=torch.uint8, device="cuda")
    a = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=61, flags=flags, ws=ws, block_rule=rule)
    assert a.iters == 61
    st = pkg.aspot_state_export(dp, ws, flags)
    assert st.t == 61 and 0.0 < st.theta < 1.0
    b = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=122, flags=flags, block_rule=rule, resume=st)
    c = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=122, flags=flags, block_rule=rule)
    assert b.iters == c.iters == 122
    np.testing.assert_array_equal(_np(b.plan.u), _np(c.plan.u))
    np.testing.assert_array_equal(_np(b.plan.v), _np(c.plan.v))
    assert float(b.plan.w.item()) == float(c.plan.w.item())
    assert b.objective == c.objective
    with pytest.raises(pkg.PotError) as e:      # a resume excludes a warm start
        pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=122, resume=st, u0=b.plan.u)
    assert e.value.status == 1
