"""GPU test of pot_marginals_static, the entry point for callers that cannot
allocate device memory (its scratch lives in a fixed array inside the
library).  It must give the same log row / column sums as pot_marginals with a
caller workspace, call after call, even though every call reuses the same
array; and it must refuse a problem too large for the array before launching
anything.  (Collected last on purpose: a failure here leaves every other test
already run.)"""
import ctypes as ct

import numpy as np
import pytest
import torch

import paper_2601_17196_gb300 as pkg
import pot_workloads as W
from oracle import pot as O
from paper_2601_17196_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _call_static(dp, gamma, u, v, w):
    f = B.lib().pot_marginals_static
    f.argtypes = [ct.POINTER(B._Problem), ct.c_double, ct.c_void_p, ct.c_void_p, ct.c_double,
                  ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
    f.restype = ct.c_int
    lrow = torch.full((dp.n,), float("nan"), dtype=torch.float64, device="cuda")
    lcol = torch.full((dp.m,), float("nan"), dtype=torch.float64, device="cuda")
    tot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = f(ct.byref(dp.struct()), gamma, u.data_ptr(), v.data_ptr(), float(w), lrow.data_ptr(), lcol.data_ptr(),
           tot.data_ptr(), ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, lrow.cpu().numpy(), lcol.cpu().numpy(), float(tot.item())


def _close(a, b):
    # the tolerance of the per-pass parity tests: 5e-6 + 2e-7 |log-sum|
    return np.all(np.abs(a - b) <= 5e-6 + 2e-7 * np.abs(b))


def test_static_scratch_matches_workspace_entry_point_two_calls_in_a_row():
    # call 1: dense FP32 cost (CUDA-core pass); call 2: BF16 points (tcgen05 pass)
    p1 = W.small_dense(1, n=300, m=457)
    p2 = W.cloud_32k(3, n=385, m=521)
    p2.cost_scale = 1.0 / O.sqeuclid_cost(p2.X, p2.Y, 1.0).max()
    rng = np.random.default_rng(5)
    for pb, gam in ((p1, 0.02), (p2, 0.02), (p1, 0.05)):
        dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
        u = torch.tensor(rng.uniform(-20, 2, dp.n), device="cuda")
        v = torch.tensor(rng.uniform(-20, 2, dp.m), device="cuda")
        w = 1.5
        st, lr, lc, tot = _call_static(dp, gam, u, v, w)
        assert st == 0, B.lib().pot_last_error()
        er, ec, etot = pkg.pot_marginals(dp, gam, u, v, w)
        er, ec = er.cpu().numpy(), ec.cpu().numpy()
        assert _close(lr, er) and _close(lc, ec)
        assert abs(np.log(tot) - np.log(etot)) <= 5e-6 + 2e-7 * abs(np.log(etot))


def _pts_problem(n, m, seed=0):
    g = torch.Generator().manual_seed(seed)
    X = torch.rand(n, 3, generator=g).cuda()
    Y = torch.rand(m, 3, generator=g).cuda()
    r = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    c = torch.full((m,), 1.2 / m, dtype=torch.float64, device="cuda")
    return pkg.DeviceProblem(pkg.COST_SQEUCLID_F32, r, c, 0.8, X=X, Y=Y, cost_scale=20.0)


def test_static_scratch_bound_is_the_pass_scratch_just_under_and_just_over():
    """The size check counts what the pass itself needs
    (pot_marginals_workspace_size), not the solvers' larger workspace: the
    largest square problem that fits runs and matches pot_marginals, one row
    more is refused with POT_ENOMEM before anything is launched."""
    limit = 16 << 20
    lo, hi = 1000, 60000
    assert pkg.marginals_workspace_bytes(_pts_problem(lo, lo)) <= limit
    assert pkg.marginals_workspace_bytes(_pts_problem(hi, hi)) > limit
    while hi - lo > 1:                        # largest n with n x n fitting (host-side queries only)
        mid = (lo + hi) // 2
        if pkg.marginals_workspace_bytes(_pts_problem(mid, mid)) <= limit:
            lo = mid
        else:
            hi = mid
    fit = _pts_problem(lo, lo, seed=1)
    assert pkg.workspace_bytes(fit) > limit   # the old whole-solver bound would have refused it
    u = torch.linspace(-3.0, 1.0, lo, dtype=torch.float64, device="cuda")
    v = torch.linspace(-2.0, 0.5, lo, dtype=torch.float64, device="cuda")
    st, lr, lc, tot = _call_static(fit, 0.05, u, v, 0.25)
    assert st == 0, B.lib().pot_last_error()
    er, ec, etot = pkg.pot_marginals(fit, 0.05, u, v, 0.25)
    assert _close(lr, er.cpu().numpy()) and _close(lc, ec.cpu().numpy())
    over = _pts_problem(hi, hi)                # hi = lo + 1
    assert pkg.marginals_workspace_bytes(over) > limit
    u2 = torch.zeros(over.n, dtype=torch.float64, device="cuda")
    v2 = torch.zeros(over.m, dtype=torch.float64, device="cuda")
    st, lr, lc, tot = _call_static(over, 0.05, u2, v2, 0.0)
    assert st == 2
    assert b"16 MiB" in B.lib().pot_last_error()
    assert np.isnan(lr).all() and np.isnan(lc).all()      # nothing was launched
