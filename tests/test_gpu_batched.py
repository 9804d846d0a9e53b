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
    res = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=5000)
    for pb, dp, r in zip(insts, probs, res):
        C = O.sqeuclid_cost(pb.X, pb.Y, 0.0)
        conv = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=5000)
        assert r.status == 0 and r.err_final <= r.eps_stop
        assert abs(r.iters - conv.iters) <= 2      # the stop test may flip on a near-tie of E_t
        # same number of iterations in the oracle: the iterates (and objectives) agree
        ora = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=r.iters, no_stop=True)
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
