"""GPU parity of the tcgen05 on-the-fly squared-Euclidean path (BF16 points,
d a multiple of 64) against the FP64 oracle, and against the CUDA-core path.

Tolerances: the dot products come from BF16 x BF16 products accumulated in
FP32 by the tensor cores; the normalised cost then carries an absolute error
of about 1e-7 and the logit (cost / gamma, gamma = 0.02) about 1e-5 / ln 2 in
the worst case, so per-pass log-sums are checked to 3e-5, solver potentials to
2e-4 (1 + |u|) and objectives to 1e-5 relative.
"""
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


def _cloud(seed, n, m, d=128):
    pb = W.cloud_32k(seed, n=n, m=m, d=d)
    Dm = O.sqeuclid_cost(pb.X, pb.Y, 1.0)
    pb.cost_scale = 1.0 / Dm.max()
    return pb, Dm


@pytest.mark.parametrize("n,m,d", [(128, 128, 128), (385, 521, 128), (1000, 1301, 64), (77, 900, 256), (1, 3, 128)])
def test_tc_marginals_match_oracle(n, m, d):
    pb, Dm = _cloud(n + m, n, m, d)
    C = Dm * pb.cost_scale
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    rng = np.random.default_rng(1)
    gam = 0.02
    for spread in (5.0, 60.0):
        u, v, w = rng.uniform(-spread, 1, n), rng.uniform(-spread, 1, m), 2.0
        lr, lc, tot = pkg.pot_marginals(dp, gam, _t(u), _t(v), w)
        L = O.log_gibbs(C, gam, u, v, w)
        er, ec = O.logsumexp(L, axis=1), O.logsumexp(L, axis=0)
        assert np.abs(_np(lr) - er).max() <= 3e-5 + 2e-7 * np.abs(er).max()
        assert np.abs(_np(lc) - ec).max() <= 3e-5 + 2e-7 * np.abs(ec).max()
    assert pkg.pot_cost_max(dp) == pytest.approx(Dm.max(), rel=1e-5)


def test_tc_round_and_objective_match_oracle():
    pb, Dm = _cloud(5, 300, 420)
    C = Dm * pb.cost_scale
    ora = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=30, no_stop=True)
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    plan, branch = pkg.pot_round(dp, pb.gamma, _t(ora.z.u), _t(ora.z.v), ora.z.w)
    Xo = O.round_pot(O.primal_plan(C, pb.gamma, ora.z), pb.r, pb.c, pb.s)
    f, g, p, q = _np(plan.f), _np(plan.g), _np(plan.p), _np(plan.q)
    X = np.exp(f[:, None] + g[None, :] - C / pb.gamma) + float(plan.kappa.item()) * np.outer(p, q)
    np.testing.assert_allclose(X, Xo, rtol=0, atol=2e-4 * Xo.max())
    obj = pkg.pot_objective(dp, plan, pb.gamma)
    assert obj == pytest.approx(O.objective(C, Xo), rel=1e-4)
    assert obj == pytest.approx(O.objective(C, X), rel=1e-5)


def test_tc_fixed_iterations_match_oracle_and_simt():
    pb, Dm = _cloud(7, 256, 320)
    C = Dm * pb.cost_scale
    K = 30
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    flags = pkg.FLAG_NO_STOP | pkg.FLAG_TRACE
    tc = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=K, flags=flags, check_every=6)
    si = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=K, flags=flags | pkg.FLAG_FORCE_SIMT, check_every=6)
    took = tc.trace[:, 3] > 0.5
    ora = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=K, no_stop=True, forced_hat=took)
    for res in (tc, si):
        u, v = _np(res.plan.u), _np(res.plan.v)
        np.testing.assert_allclose(u, ora.z.u, rtol=0, atol=2e-4 * (1 + np.abs(ora.z.u).max()))
        np.testing.assert_allclose(v, ora.z.v, rtol=0, atol=2e-4 * (1 + np.abs(ora.z.v).max()))
    assert tc.objective == pytest.approx(si.objective, rel=1e-5)


def test_tc_greedy_fixed_iterations_match_oracle():
    """Greedy block rule on the tcgen05 pass (several tiles, ragged edges):
    the oracle replays the GPU's argmin and block decisions."""
    pb, Dm = _cloud(9, 300, 420)
    C = Dm * pb.cost_scale
    K = 30
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    res = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=K, flags=pkg.FLAG_NO_STOP | pkg.FLAG_TRACE,
                          check_every=6, block_rule=pkg.BLOCK_GREEDY)
    code = np.rint(res.trace[:, 3]).astype(np.int64)
    took, k, k2 = (code & 1) > 0, (code >> 1) & 3, (code >> 3) & 3
    ora = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=K, no_stop=True, forced_hat=took,
                  forced_blocks=list(zip(k, k2)), block_rule="greedy")
    u, v = _np(res.plan.u), _np(res.plan.v)
    np.testing.assert_allclose(u, ora.z.u, rtol=0, atol=2e-4 * (1 + np.abs(ora.z.u).max()))
    np.testing.assert_allclose(v, ora.z.v, rtol=0, atol=2e-4 * (1 + np.abs(ora.z.v).max()))
    assert float(res.plan.w.item()) == pytest.approx(ora.z.w, abs=2e-4 * (1 + abs(ora.z.w)))


def test_profiled_solve_times_every_pass():
    """POT_FLAG_PROFILE: every main-loop pass timed, results unchanged."""
    pb, Dm = _cloud(11, 200, 260)
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    a = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=40, flags=pkg.FLAG_NO_STOP | pkg.FLAG_PROFILE, check_every=9)
    b = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=40, flags=pkg.FLAG_NO_STOP, check_every=9)
    # three timed passes per iteration, two when k = t mod 3 = 2 (the w-step's
    # closed form replaces the pass at z^t; its fallback pass is not timed)
    assert a.pass_launches == sum(2 if t % 3 == 2 else 3 for t in range(40)) and a.pass_ms > 0
    assert a.kernel_launches >= 40 * 10
    np.testing.assert_array_equal(_np(a.plan.u), _np(b.plan.u))
    assert a.objective == b.objective


def _rows_lse(X, Y, rows, cs, gamma, u, v, w):
    """Oracle log-sums of sampled rows (and, transposed, columns) of B at full size."""
    out = np.empty(len(rows))
    for k, i in enumerate(rows):
        c = cs * ((X[i][None, :] - Y) ** 2).sum(axis=1)
        out[k] = O.logsumexp(u[i] + v + w - c / gamma)
    return out


@pytest.mark.parametrize("n,m,d", [(9000, 8300, 128), (8193, 9001, 64)])
def test_columns_only_pass_runs_transposed(n, m, d):
    """Above 32 row blocks of 256 a columns-only pass runs as the rows-only
    kernel on the transposed problem (Y as the row operand): its column sums
    against the oracle on sampled columns, against the two-sided pass on all
    columns, and the mass summed over the columns."""
    pb = W.cloud_32k(11, n=n, m=m, d=d)
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    X, Y = W.from_bf16_bits(pb.X_bf16), W.from_bf16_bits(pb.Y_bf16)
    g = np.random.default_rng(n)
    cols = np.sort(g.choice(m, 128, replace=False))
    cs, gam = 1.0 / 4000.0, 0.02
    dp.cost_scale = cs
    for lo, hi in ((-14.0, -10.0), (-60.0, -5.0)):
        u, v, w = g.uniform(lo, hi, n), g.uniform(lo, hi, m), 3.0
        none, lcc, totc = pkg.pot_marginals(dp, gam, _t(u), _t(v), w, rows=False)
        assert none is None
        lr, lc, tot = pkg.pot_marginals(dp, gam, _t(u), _t(v), w)
        ec = _rows_lse(Y, X, cols, cs, gam, v, u, w)
        assert np.abs(_np(lcc)[cols] - ec).max() <= 3e-5 + 2e-7 * np.abs(ec).max()
        assert np.abs(_np(lcc) - _np(lc)).max() <= 3e-5 + 2e-7 * np.abs(_np(lc)).max()
        assert totc == pytest.approx(tot, rel=3e-5)


def test_transposed_column_passes_in_the_loop_match_simt():
    """ASPOT at n = 9000 (cyclic rule: the pass at z^t after a u-step is
    columns-only and runs transposed at this size), 30 fixed iterations
    against the CUDA-core path: potentials within 2e-4 (1 + |u|)."""
    pb = W.cloud_32k(12, n=9000, m=8800)
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    K = 30
    a = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=K, flags=pkg.FLAG_NO_STOP)
    b = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=K, flags=pkg.FLAG_NO_STOP | pkg.FLAG_FORCE_SIMT)
    assert a.iters == b.iters == K and a.status == b.status == 0
    for x, y in ((_np(a.plan.u), _np(b.plan.u)), (_np(a.plan.v), _np(b.plan.v))):
        np.testing.assert_allclose(x, y, rtol=0, atol=2e-4 * (1 + np.abs(y).max()))
    assert a.err_final == pytest.approx(b.err_final, rel=2e-2)


def test_cloud_32k_full_size_sampled():
    """The bench's workload at its full size (n = m = 32768, d = 128 BF16) in the
    launch configuration the bench times: (1) one fused pass with given
    potentials, 256 sampled rows and 256 sampled columns against the oracle in
    FP64; (2) a whole solve, whose rounded plan is checked for feasibility on
    sampled rows and columns in FP64 and whose E_t meets the threshold."""
    pb = W.cloud_32k(0)
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    X, Y = W.from_bf16_bits(pb.X_bf16), W.from_bf16_bits(pb.Y_bf16)
    n, m = X.shape[0], Y.shape[0]
    g = np.random.default_rng(5)
    rows = np.sort(g.choice(n, 256, replace=False))
    cols = np.sort(g.choice(m, 256, replace=False))
    # (1) one pass with an explicit cost scale (an input, like the potentials)
    cs, gam = 1.0 / 4000.0, pb.gamma
    u, v, w = g.uniform(-14, -10, n), g.uniform(-14, -10, m), 3.0
    dp.cost_scale = cs
    lr, lc, _ = pkg.pot_marginals(dp, gam, _t(u), _t(v), w)
    er = _rows_lse(X, Y, rows, cs, gam, u, v, w)
    ec = _rows_lse(Y, X, cols, cs, gam, v, u, w)
    assert np.abs(_np(lr)[rows] - er).max() <= 3e-5 + 2e-7 * np.abs(er).max()
    assert np.abs(_np(lc)[cols] - ec).max() <= 3e-5 + 2e-7 * np.abs(ec).max()
    # the columns-only pass of the solve's loop (transposed at this size)
    _, lcc, _ = pkg.pot_marginals(dp, gam, _t(u), _t(v), w, rows=False)
    assert np.abs(_np(lcc)[cols] - ec).max() <= 3e-5 + 2e-7 * np.abs(ec).max()
    # (2) the solve the bench times (cost normalised by its maximum, computed on the GPU)
    dp.cost_scale = 0.0
    res = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=20000)
    assert res.status == 0 and res.err_final <= res.eps_stop and res.nonfinite == 0
    assert res.mass == pytest.approx(pb.s)
    f, gg, p, q = (_np(t) for t in (res.plan.f, res.plan.g, res.plan.p, res.plan.q))
    kap = float(res.plan.kappa.item())
    csr = res.cost_scale
    for i in rows[:64]:
        c = csr * ((X[i][None, :] - Y) ** 2).sum(axis=1)
        xi = np.exp(f[i] + gg - c / res.gamma).sum() + kap * p[i] * q.sum()
        assert xi <= pb.r[i] * (1 + 1e-5) + 1e-15
    for j in cols[:64]:
        c = csr * ((Y[j][None, :] - X) ** 2).sum(axis=1)
        xj = np.exp(f + gg[j] - c / res.gamma).sum() + kap * p.sum() * q[j]
        assert xj <= pb.c[j] * (1 + 1e-5) + 1e-15


def test_cloud_32k_full_size_greedy_solve():
    """The greedy-block-rule solve the bench times beside the headline (same
    workload, n = m = 32768, d = 128 BF16): it reaches the threshold in fewer
    iterations than the cyclic rule, and its rounded plan is feasible in FP64
    on sampled rows and columns with total mass s."""
    pb = W.cloud_32k(0)
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    X, Y = W.from_bf16_bits(pb.X_bf16), W.from_bf16_bits(pb.Y_bf16)
    n, m = X.shape[0], Y.shape[0]
    g = np.random.default_rng(6)
    rows = np.sort(g.choice(n, 64, replace=False))
    cols = np.sort(g.choice(m, 64, replace=False))
    res = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=20000, block_rule=pkg.BLOCK_GREEDY)
    assert res.status == 0 and res.err_final <= res.eps_stop and res.nonfinite == 0
    assert res.iters < 2000                       # the cyclic rule needs 2261 on this workload
    assert res.mass == pytest.approx(pb.s)
    f, gg, p, q = (_np(t) for t in (res.plan.f, res.plan.g, res.plan.p, res.plan.q))
    kap = float(res.plan.kappa.item())
    csr = res.cost_scale
    for i in rows:
        c = csr * ((X[i][None, :] - Y) ** 2).sum(axis=1)
        xi = np.exp(f[i] + gg - c / res.gamma).sum() + kap * p[i] * q.sum()
        assert xi <= pb.r[i] * (1 + 1e-5) + 1e-15
    for j in cols:
        c = csr * ((Y[j][None, :] - X) ** 2).sum(axis=1)
        xj = np.exp(f + gg[j] - c / res.gamma).sum() + kap * p.sum() * q[j]
        assert xj <= pb.c[j] * (1 + 1e-5) + 1e-15


@pytest.mark.parametrize("d", [128, 3])
def test_sinkhorn_on_point_clouds_matches_oracle(d):
    """The feasible Sinkhorn baseline on point clouds: BF16 d = 128 through the
    tcgen05 pass, FP32 d = 3 through the CUDA-core pass.  Iterations within one
    of the oracle's, objective to 1e-5 relative (the tcgen05 pass's log-sum
    error is a few 1e-6), feasible rounded plan."""
    if d == 128:
        pb, Dm = _cloud(13, 300, 420)
    else:
        rng = np.random.default_rng(14)
        X = rng.uniform(0, 1, (300, 3)).astype(np.float32).astype(np.float64)
        Y = rng.uniform(0, 1, (420, 3)).astype(np.float32).astype(np.float64)
        pb = W.Problem("pts", np.full(300, 1.0 / 300), np.full(420, 1.25 / 420), 0.9, 0.05, 1e-3, X=X, Y=Y)
        Dm = O.sqeuclid_cost(X, Y, 1.0)
        pb.cost_scale = 1.0 / Dm.max()
    C = Dm * pb.cost_scale
    kind = pkg.COST_SQEUCLID_BF16 if d == 128 else pkg.COST_SQEUCLID_F32
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda", kind=kind)
    res = pkg.sinkhorn_pot_solve(dp, pb.gamma, pb.eps, max_iter=20000)
    ora = O.solve_sinkhorn(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=20000)
    assert res.status == 0 and abs(res.iters - ora.iters) <= 1
    assert abs(res.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    f, g, p, q = (_np(t) for t in (res.plan.f, res.plan.g, res.plan.p, res.plan.q))
    X = np.exp(f[:, None] + g[None, :] - C / res.gamma) + float(res.plan.kappa.item()) * np.outer(p, q)
    # rows the rounding makes tight meet r exactly in the GPU's own arithmetic; the
    # plan re-evaluated in FP64 differs by the pass's log-sum error (a few 1e-6 on
    # the tcgen05 pass, whose products accumulate in FP32), so 1e-5 there
    tol = 1e-5 if d == 128 else 1e-6
    assert (X.sum(1) <= pb.r * (1 + tol)).all() and (X.sum(0) <= pb.c * (1 + tol)).all()
    assert X.sum() == pytest.approx(pb.s, rel=tol)
