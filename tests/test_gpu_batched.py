"""GPU parity of the batched solver (many uneven 3-D instances in lockstep)
against the FP64 oracle, instance by instance, and against single solves."""
import numpy as np
import pytest

import paper_2601_17196_gb300 as pkg
import pot_workloads as W
from oracle import pot as O

pytestmark = pytest.mark.gpu


def test_batched_matches_oracle_and_single_solves():
    insts = W.batch_3d(seed=4, count=6, nmin=64, nmax=520)
    probs = [pkg.DeviceProblem.from_workload(pb, device="cuda") for pb in insts]
    res = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=5000, decisions=True)
    for pb, dp, r in zip(insts, probs, res):
        C = O.sqeuclid_cost(pb.X, pb.Y, 0.0)
        conv = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=5000)
        assert r.status == 0 and r.err_final <= r.eps_stop
        # E_t is not monotone near the threshold: the summation order (tile shape)
        # can move its first crossing by a few iterations
        assert abs(r.iters - conv.iters) <= 4
        # same number of iterations in the oracle, with the batched solve's argmin
        # decisions replayed (a near-tie of phi(z^) against phi(z_check) may go the
        # other way in FP32, as for the single solve below): the objectives agree
        assert r.iters <= len(r.decisions)
        ora = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=r.iters, no_stop=True,
                            forced_hat=list((r.decisions & 1) > 0))
        assert abs(r.objective - ora.objective) <= 1e-5 * abs(ora.objective)
        single = pkg.aspot_solve(dp, 0.05, 1e-3, max_iter=5000, flags=pkg.FLAG_TRACE)
        # E_t is not monotone near the threshold: rounding-level differences between
        # the two programs move its first crossing by a few iterations
        assert single.status == 0 and single.err_final <= single.eps_stop
        assert abs(single.iters - conv.iters) <= 4 and abs(single.iters - r.iters) <= 4
        # the single solve against the oracle with its own argmin decisions replayed
        # (a near-tie of phi(z^) against phi(z_check) may go the other way in FP32)
        took = single.trace[:, 3] > 0.5
        ora_s = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=single.iters, no_stop=True,
                              forced_hat=list(took))
        assert abs(single.objective - ora_s.objective) <= 1e-5 * abs(ora_s.objective)
        f, g, p, q = (t.cpu().numpy() for t in (r.plan.f, r.plan.g, r.plan.p, r.plan.q))
        X = np.exp(f[:, None] + g[None, :] - C / r.gamma) + float(r.plan.kappa.item()) * np.outer(p, q)
        assert (X.sum(1) <= pb.r * (1 + 1e-6)).all() and (X.sum(0) <= pb.c * (1 + 1e-6)).all()
        assert X.sum() == pytest.approx(pb.s, rel=1e-6)


def test_batched_fixed_iterations_and_invalid_mix():
    insts = W.batch_3d(seed=5, count=3, nmin=64, nmax=300)
    probs = [pkg.DeviceProblem.from_workload(pb, device="cuda") for pb in insts]
    res = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=30, flags=pkg.FLAG_NO_STOP, check_every=6)
    for pb, r in zip(insts, res):
        C = O.sqeuclid_cost(pb.X, pb.Y, 0.0)
        ora = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=30, no_stop=True)
        assert r.iters == 30
        np.testing.assert_allclose(r.plan.u.cpu().numpy(), ora.z.u, rtol=0, atol=2e-5 * (1 + np.abs(ora.z.u).max()))
    bad = list(probs)
    bad[1] = pkg.DeviceProblem(pkg.COST_SQEUCLID_BF16, probs[1].r, probs[1].c, probs[1].s,
                               X=probs[1].X.bfloat16(), Y=probs[1].Y.bfloat16())
    with pytest.raises(pkg.PotError) as e:
        pkg.aspot_solve_batched(bad, 0.05, 1e-3)
    assert e.value.status == 1


def _batch_probs(seed, count, nmin, nmax):
    insts = W.batch_3d(seed=seed, count=count, nmin=nmin, nmax=nmax)
    return insts, [pkg.DeviceProblem.from_workload(pb, device="cuda") for pb in insts]


def test_batched_every_tile_shape_matches_default():
    """Each candidate tile shape of the autotuner (pinned through the cache)
    follows the default 256 x 256 tiles' iterates: the shape only changes the
    FP32 summation order of the partials.  60 fixed iterations agree to the
    parity tolerance, and every shape solves every instance to its threshold
    (where E_t is not monotone, so its first crossing may move by a few
    iterations)."""
    insts, probs = _batch_probs(8, 10, 64, 900)
    K = 60
    base = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=K, flags=pkg.FLAG_NO_STOP, check_every=6)
    assert all(r.tile_rows == 256 and r.tile_cols == 256 for r in base)
    ub = [r.plan.u.cpu().numpy() for r in base]
    vb = [r.plan.v.cpu().numpy() for r in base]
    for H in (32, 64, 128, 256):
        for Wc in (128, 256):
            pkg.autotune_clear()
            pkg.autotune_set(probs, H, Wc)
            res = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=K, flags=pkg.FLAG_NO_STOP | pkg.FLAG_AUTOTUNE,
                                          check_every=6)
            for k, r in enumerate(res):
                assert (r.tile_rows, r.tile_cols) == (H, Wc) and r.tune_ms == 0.0 and r.iters == K
                np.testing.assert_allclose(r.plan.u.cpu().numpy(), ub[k], rtol=0, atol=2e-5 * (1 + np.abs(ub[k]).max()))
                np.testing.assert_allclose(r.plan.v.cpu().numpy(), vb[k], rtol=0, atol=2e-5 * (1 + np.abs(vb[k]).max()))
            conv = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=5000, flags=pkg.FLAG_AUTOTUNE)
            assert all(r.status == 0 and r.err_final <= r.eps_stop for r in conv)
    pkg.autotune_clear()


def test_batched_autotune_times_candidates_then_caches():
    insts, probs = _batch_probs(9, 40, 64, 2048)
    pkg.autotune_clear()
    first = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=5000, flags=pkg.FLAG_AUTOTUNE)
    shape = (first[0].tile_rows, first[0].tile_cols)
    assert shape[0] in (32, 64, 128, 256) and shape[1] in (128, 256)
    assert first[0].tune_ms > 0.0
    assert pkg.autotune_lookup(probs) == shape
    again = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=5000, flags=pkg.FLAG_AUTOTUNE)
    assert (again[0].tile_rows, again[0].tile_cols) == shape and again[0].tune_ms == 0.0
    for pb, r in zip(insts[:5], again[:5]):
        C = O.sqeuclid_cost(pb.X, pb.Y, 0.0)
        ora = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=r.iters, no_stop=True)
        assert r.status == 0
        assert abs(r.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    pkg.autotune_clear()


def _replay(codes):
    codes = np.asarray(codes, dtype=np.int64)
    return list((codes & 1) > 0), list(zip((codes >> 1) & 3, (codes >> 3) & 3))


def test_batched_greedy_rule_matches_oracle():
    """Greedy block rule in the batched solver, with the oracle replaying each
    instance's recorded argmin and block decisions (pot_trace_batched): 30
    fixed iterations match in the potentials, converged solves in the
    objective at the GPU's iteration count, and every instance reaches its
    threshold in fewer iterations than the cyclic rule."""
    insts, probs = _batch_probs(11, 5, 64, 400)
    K = 30
    res = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=K, flags=pkg.FLAG_NO_STOP, check_every=6,
                                  block_rule=pkg.BLOCK_GREEDY, decisions=True)
    for pb, r in zip(insts, res):
        C = O.sqeuclid_cost(pb.X, pb.Y, 0.0)
        assert r.iters == K and len(r.decisions) == K
        took, blocks = _replay(r.decisions)
        ora = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=K, no_stop=True, block_rule="greedy",
                      forced_hat=took, forced_blocks=blocks)
        np.testing.assert_allclose(r.plan.u.cpu().numpy(), ora.z.u, rtol=0, atol=2e-5 * (1 + np.abs(ora.z.u).max()))
        np.testing.assert_allclose(r.plan.v.cpu().numpy(), ora.z.v, rtol=0, atol=2e-5 * (1 + np.abs(ora.z.v).max()))
    conv = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=5000, block_rule=pkg.BLOCK_GREEDY, decisions=True)
    cyc = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=5000)
    for pb, r, c in zip(insts, conv, cyc):
        assert r.status == 0 and r.err_final <= r.eps_stop
        assert r.iters < c.iters                      # the greedy rule needs fewer iterations here
        C = O.sqeuclid_cost(pb.X, pb.Y, 0.0)
        took, blocks = _replay(r.decisions)
        ora = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=r.iters, no_stop=True,
                            block_rule="greedy", forced_hat=took, forced_blocks=blocks)
        assert abs(r.objective - ora.objective) <= 1e-5 * abs(ora.objective)
        f, g, p, q = (t.cpu().numpy() for t in (r.plan.f, r.plan.g, r.plan.p, r.plan.q))
        X = np.exp(f[:, None] + g[None, :] - C / r.gamma) + float(r.plan.kappa.item()) * np.outer(p, q)
        assert (X.sum(1) <= pb.r * (1 + 1e-6)).all() and (X.sum(0) <= pb.c * (1 + 1e-6)).all()
        assert X.sum() == pytest.approx(pb.s, rel=1e-6)


def test_batched_records_cyclic_decisions():
    """The cyclic rule's recorded blocks are t mod 3 (k2 = k), and replaying
    the recorded argmin decisions reproduces the oracle's iterates."""
    insts, probs = _batch_probs(12, 4, 64, 300)
    K = 24
    res = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=K, flags=pkg.FLAG_NO_STOP, check_every=6,
                                  decisions=True)
    for pb, r in zip(insts, res):
        took, blocks = _replay(r.decisions)
        assert blocks == [(t % 3, t % 3) for t in range(K)]
        C = O.sqeuclid_cost(pb.X, pb.Y, 0.0)
        ora = O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=K, no_stop=True, forced_hat=took)
        np.testing.assert_allclose(r.plan.u.cpu().numpy(), ora.z.u, rtol=0, atol=2e-5 * (1 + np.abs(ora.z.u).max()))
