"""GPU tests of the single-cluster ASPOT loop (small problems, CUDA-core passes).

Problems of at most 2^18 cost entries iterate in one thread-block cluster:
the CTAs share each pass's tiles and CTA 0 runs the update of the block rule
(Algorithm 2 with the Greenkhorn couplings of Algorithm 1) on the solver's own
vectors, one launch per check_every iterations.  These tests hold it to the
same bars as the staged loop (separate kernels in CUDA graphs, forced with
FLAG_STAGED):
  * converged solves: E_t below the threshold, objective within 1e-5
    relative of the FP64 oracle run for the same number of iterations with the
    loop's recorded decisions, within 2e-4 of the staged loop's own solve (each
    stops at the first iterate below the threshold, which rounding can move
    by a few iterations), the rounded plan feasible in FP64;
  * against the staged loop on the same instance: the same iteration count
    within one, potentials within 2e-5 (1 + |u|) after 60 fixed iterations
    (both are FP32 passes with FP64 updates; the cluster loop takes the sums at
    z^t from a full pass where the staged loop uses closed forms, so they agree
    to rounding, not bit for bit);
  * checkpoint / resume through the cluster loop, bit for bit;
  * ragged and degenerate shapes, warm starts, max_iter.
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


def _points(n, m, d, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, d)).astype(np.float32).astype(np.float64)
    Y = (rng.uniform(0, 1, (m, d)) * 0.8 + 0.1).astype(np.float32).astype(np.float64)
    r, c = np.full(n, 1.0 / n), np.full(m, 1.25 / m)
    pb = W.Problem("pts", r, c, 0.8, 0.05, 1e-3, X=X, Y=Y)
    Dm = O.sqeuclid_cost(X, Y, 1.0)
    pb.cost_scale = 1.0 / Dm.max()
    return pb, Dm * pb.cost_scale


CASES = [("dense", 256, 256), ("dense", 300, 257), ("dense", 500, 520), ("dense", 7, 300),
         ("dense", 513, 129), ("points", 500, 400), ("points", 130, 1000)]


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("src,n,m", CASES)
def test_cluster_loop_converges_like_the_oracle(src, n, m, rule):
    if src == "dense":
        pb = W.small_dense(5, n=n, m=m)
        C = pb.C.astype(np.float64)
        dp, cmax = _dev(pb), None
    else:
        pb, C = _points(n, m, 2, 40 + n)
        dp, cmax = _dev(pb, kind=pkg.COST_SQEUCLID_F32), 1.0
    res = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=5000, block_rule=rule, flags=pkg.FLAG_TRACE)
    assert res.cluster_loop == 1
    assert res.status == 0 and res.err_final <= res.eps_stop
    stg = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=5000, block_rule=rule, flags=pkg.FLAG_STAGED)
    assert stg.cluster_loop == 0 and stg.status == 0
    # one launch per 24 iterations (plus the set-up, rounding and objective kernels)
    assert res.kernel_launches < stg.kernel_launches / 4
    # Both stop at the first iterate with E_t <= eps~.  The two loops round
    # differently (sums at z^t from a pass instead of closed forms, block sums
    # in another order), which moves that iterate by a few iterations (more for
    # the greedy rule, whose choices near convergence are near-ties) and the
    # plan's objective by up to ~1e-4 relative: still ten times inside the
    # accuracy eps = 1e-3 (about 1.3 % of these objectives) both plans carry.
    assert abs(res.iters - stg.iters) <= max(3, 0.1 * stg.iters if rule else 0.03 * stg.iters)
    assert abs(res.objective - stg.objective) <= 2e-4 * abs(stg.objective)
    # the oracle's FP64 run of the same number of iterations with the loop's
    # recorded decisions replayed (argmin near-ties can go either way in FP32):
    # the 1e-5 bar
    code = np.rint(res.trace[:, 3]).astype(np.int64)
    kw = {} if cmax is None else {"cmax": cmax}
    if rule:
        kw.update(block_rule="greedy", forced_blocks=list(zip((code >> 1) & 3, (code >> 3) & 3)))
    ora = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=res.iters, no_stop=True,
                        forced_hat=list((code & 1) > 0), **kw)
    assert abs(res.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    X = _plan_fp64(C, res.plan, res.gamma, 1.0 if cmax else res.cost_scale)
    _check_feasible(X, pb.r, pb.c, pb.s)


@pytest.mark.parametrize("rule", [0, 1])
def test_cluster_loop_fixed_iterations_match_the_staged_loop(rule):
    pb = W.small_dense(3, n=200, m=232)
    dp = _dev(pb)
    K = 60
    a = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=K, flags=pkg.FLAG_NO_STOP, block_rule=rule, check_every=9)
    b = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=K, flags=pkg.FLAG_NO_STOP | pkg.FLAG_STAGED,
                        block_rule=rule, check_every=9)
    assert a.cluster_loop == 1 and b.cluster_loop == 0
    assert a.iters == b.iters == K
    for x, y in ((_np(a.plan.u), _np(b.plan.u)), (_np(a.plan.v), _np(b.plan.v))):
        np.testing.assert_allclose(x, y, rtol=0, atol=2e-5 * (1 + np.abs(y).max()))
    wa, wb = float(a.plan.w.item()), float(b.plan.w.item())
    assert wa == pytest.approx(wb, abs=2e-5 * (1 + abs(wb)))
    assert a.err_final == pytest.approx(b.err_final, rel=1e-3, abs=1e-9)


@pytest.mark.parametrize("rule", [0, 1])
def test_cluster_loop_resume_continues_exactly(rule):
    """61 iterations, exported, resumed to 122 (block 61 mod 3 next): bit for
    bit the uninterrupted 122-iteration run of the cluster loop."""
    pb = W.small_dense(3, n=200, m=233)
    dp = _dev(pb)
    flags = pkg.FLAG_NO_STOP
    ws = torch.empty(pkg.binding.workspace_bytes(dp, flags) + 256, dtype=torch.uint8, device="cuda")
    a = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=61, flags=flags, ws=ws, block_rule=rule, check_every=12)
    assert a.cluster_loop == 1 and a.iters == 61
    st = pkg.aspot_state_export(dp, ws, flags)
    assert st.t == 61 and 0.0 < st.theta < 1.0
    b = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=122, flags=flags, block_rule=rule, resume=st)
    c = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=122, flags=flags, block_rule=rule)
    assert b.cluster_loop == c.cluster_loop == 1
    assert b.iters == c.iters == 122
    np.testing.assert_array_equal(_np(b.plan.u), _np(c.plan.u))
    np.testing.assert_array_equal(_np(b.plan.v), _np(c.plan.v))
    assert float(b.plan.w.item()) == float(c.plan.w.item())
    assert b.objective == c.objective


def test_cluster_loop_warm_start_and_max_iter():
    pb = W.small_dense(8, n=320, m=288)
    C = pb.C.astype(np.float64)
    dp = _dev(pb)
    cold = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=5000)
    assert cold.cluster_loop == 1 and cold.status == 0
    # a warm start at the converged duals stops within a few iterations
    warm = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=5000, u0=cold.plan.u, v0=cold.plan.v,
                           w0=float(cold.plan.w.item()))
    assert warm.cluster_loop == 1 and warm.status == 0 and warm.iters < cold.iters / 4
    z0 = O.Dual(_np(cold.plan.u), _np(cold.plan.v), float(cold.plan.w.item()))
    ora = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=warm.iters, no_stop=True, z0=z0)
    assert abs(warm.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    # max_iter below the iterations needed: ENOCONV, still a feasible plan
    with pytest.raises(pkg.PotError) as e:
        pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=5, allow_noconv=False)
    assert e.value.status == 4
    few = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=5)
    assert few.status == 4 and few.cluster_loop == 1 and few.iters == 5
    _check_feasible(_plan_fp64(C, few.plan, few.gamma, few.cost_scale), pb.r, pb.c, pb.s)


def test_cluster_loop_single_entry():
    pb = W.small_dense(2, n=1, m=1)
    res = pkg.aspot_solve(_dev(pb), pb.gamma, pb.eps, max_iter=2000)
    assert res.cluster_loop == 1 and res.status == 0
    assert res.mass == pytest.approx(pb.s)


def test_large_and_profiled_solves_stay_staged():
    pb = W.small_dense(0)
    dp = _dev(pb)
    tr = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=100, flags=pkg.FLAG_TRACE | pkg.FLAG_NO_STOP)
    assert tr.cluster_loop == 1 and tr.trace.shape == (100, 4) and np.isfinite(tr.trace).all()
    assert pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=100, flags=pkg.FLAG_PROFILE | pkg.FLAG_NO_STOP).cluster_loop == 0
    big = W.dense_4096(0, n=600, m=500)
    assert pkg.aspot_solve(_dev(big), big.gamma, big.eps, max_iter=30, flags=pkg.FLAG_NO_STOP).cluster_loop == 0
