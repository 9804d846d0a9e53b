"""GPU test of the tcgen05 passes' bounded waits.

Every pipeline wait inside the tcgen05 passes (TMA data, accumulator
hand-offs, column terms) gives up after a bound; the CTA then stops issuing
work, drains the copies and MMAs it issued itself, frees its tensor memory
and raises a flag that the host turns into POT_ETIMEOUT (a stalled pass must
never come back as POT_OK with wrong sums).

The stall is made on purpose through the test hook of pot_params: a negative
wait_limit_ns makes the hot-loop passes withhold their first accumulator
hand-off (the accumulator goes to a spare barrier nobody waits on), so the
epilogue's wait runs out after |wait_limit_ns| ns.  Nothing faults and
nothing hangs: the wait is bounded, and the kernels exit normally.  The
same workspace then runs a normal solve, which must be bit for bit the solve
of a fresh workspace."""
import numpy as np
import pytest
import torch

import paper_2601_17196_gb300 as pkg
import pot_workloads as W

pytestmark = pytest.mark.gpu


def _ws(dp):
    return torch.zeros(pkg.workspace_bytes(dp) + 256, dtype=torch.uint8, device="cuda")


def _solve(dp, pb, ws, **kw):
    return pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=60, flags=pkg.FLAG_NO_STOP, check_every=12, ws=ws, **kw)


def test_stalled_tcgen05_pass_reports_timeout_and_leaves_a_usable_context():
    pb = W.cloud_32k(6, n=2048, m=1920)
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    ws = _ws(dp)
    with pytest.raises(pkg.PotError) as e:
        _solve(dp, pb, ws, wait_limit_ns=-200_000)       # 200 us, far above any real wait of these passes
    assert e.value.status == 6
    assert "gave up waiting" in str(e.value)
    torch.cuda.synchronize()                             # the context is still usable

    after = _solve(dp, pb, ws)                           # the same workspace, no hook
    fresh = _solve(dp, pb, _ws(dp))
    assert after.status == 0 and fresh.status == 0
    assert after.iters == fresh.iters == 60
    for k in ("u", "v", "w", "f", "g", "p", "q", "kappa"):
        a = getattr(after.plan, k).cpu().numpy()
        b = getattr(fresh.plan, k).cpu().numpy()
        assert np.array_equal(a, b), k
    assert after.objective == fresh.objective


def test_positive_wait_limit_leaves_the_solve_unchanged():
    """A finite, generous bound (50 ms) changes nothing when no wait comes near it."""
    pb = W.cloud_32k(7, n=1024)
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    a = _solve(dp, pb, _ws(dp), wait_limit_ns=50_000_000)
    b = _solve(dp, pb, _ws(dp))
    assert a.status == 0 and np.array_equal(a.plan.u.cpu().numpy(), b.plan.u.cpu().numpy())
    assert a.objective == b.objective
