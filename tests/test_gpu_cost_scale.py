"""GPU tests of the cost prologue when the caller leaves cost_scale at 0, the
documented default: the library then finds max C itself (one max-cost pass)
and uses 1 / max C as the cost scale, which sets both the normalised cost and
the stop threshold eps / (8 max C) of Algorithm 2's setup.

* the dense FP32 max-cost pass against the exact maximum (a maximum of FP32
  values is exact, so the comparison is bit for bit), on ragged sizes that
  span several tiles, through both the 128-bit and the scalar load paths;
* whole ASPOT and feasible Sinkhorn solves on an unnormalised dense cost
  with cost_scale = 0, against the FP64 oracle on the normalised cost: the
  cost scale must be 1 / max C and the objective must agree to 1e-5;
* a NaN or an infinity anywhere in the cost (dense, BF16 points through the
  tcgen05 max pass, FP32 3-D points through the CUDA-core pass) must be
  rejected with POT_EINVAL before the solve starts."""
import numpy as np
import pytest
import torch

import paper_2601_17196_gb300 as pkg
import pot_workloads as W
from oracle import pot as O

pytestmark = pytest.mark.gpu


def _t(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _raw_dense(seed, n, m, scale):
    """Squared distances of the 256-point workload's clouds, times `scale`,
    stored FP32 and NOT normalised (max C far from 1)."""
    g = np.random.default_rng(seed)
    X = g.uniform(0.0, 1.0, size=(n, 2))
    Y = g.normal(0.5, 0.1, size=(m, 2))
    C = (scale * ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)).astype(np.float32)
    return C


def _dense_problem(C, r, c, s, cost_scale=0.0):
    Ct = torch.tensor(np.ascontiguousarray(C, dtype=np.float32), device="cuda")
    return pkg.DeviceProblem(pkg.COST_DENSE_F32, _t(r), _t(c), s, C=Ct, cost_scale=cost_scale)


@pytest.mark.parametrize("n,m", [(257, 300), (1000, 1536), (96, 4099), (1, 5)])
def test_dense_cost_max_is_the_exact_maximum(n, m):
    C = _raw_dense(3 + n, n, m, 3.7)
    C[n // 2, m // 3] = 11.25                      # a known maximum inside the grid
    dp = _dense_problem(C, np.full(n, 1.0 / n), np.full(m, 1.0 / m), 0.5)
    got = pkg.pot_cost_max(dp)
    assert got == float(C.max()) == 11.25


def test_dense_cost_max_strided_rows():
    """ldc > m (a row-padded cost): the padding must not enter the maximum."""
    n, m, ld = 300, 250, 260
    C = _raw_dense(9, n, m, 2.0)
    Cp = np.full((n, ld), 1.0e6, dtype=np.float32)
    Cp[:, :m] = C
    Ct = torch.tensor(Cp, device="cuda")[:, :m]
    dp = pkg.DeviceProblem(pkg.COST_DENSE_F32, _t(np.full(n, 1.0 / n)), _t(np.full(m, 1.0 / m)), 0.5, C=Ct,
                           cost_scale=0.0)
    assert pkg.pot_cost_max(dp) == float(C.max())


def test_aspot_with_computed_cost_scale_matches_oracle():
    n, m = 200, 233
    C = _raw_dense(17, n, m, 5.0)
    cmax = float(C.max())
    Cn = C.astype(np.float64) / cmax                 # what cost_scale = 1 / max C means
    r, c, s = np.full(n, 1.0 / n), np.full(m, 1.2 / m), 0.8
    gamma, eps = 0.05, 1e-3
    dp = _dense_problem(C, r, c, s)
    res = pkg.aspot_solve(dp, gamma, eps, max_iter=20000, flags=pkg.FLAG_TRACE)
    assert res.status == 0
    assert res.cost_scale == 1.0 / cmax
    # stop threshold eps / (8 max C_eff) with max C_eff = 1
    assert res.eps_stop == pytest.approx(eps / 8.0, rel=1e-15)
    took = res.trace[:, 3] > 0.5
    ora = O.solve_aspot(Cn, r, c, s, eps, gamma, max_iter=res.iters, no_stop=True, forced_hat=list(took),
                        cmax=1.0)
    assert abs(res.objective - ora.objective) <= 1e-5 * abs(ora.objective)
    z = ora.solve.z
    u = res.plan.u.cpu().numpy()
    assert np.abs(u - z.u).max() <= 2e-5 * (1 + np.abs(z.u).max())


def test_sinkhorn_with_computed_cost_scale_matches_oracle():
    n, m = 180, 150
    C = _raw_dense(23, n, m, 0.37)
    cmax = float(C.max())
    Cn = C.astype(np.float64) / cmax
    r, c, s = np.full(n, 1.0 / n), np.full(m, 1.2 / m), 0.8
    dp = _dense_problem(C, r, c, s)
    res = pkg.sinkhorn_pot_solve(dp, 0.05, 1e-3, max_iter=20000)
    ora = O.solve_sinkhorn(Cn, r, c, s, 1e-3, 0.05, max_iter=20000)
    assert res.status == 0 and res.cost_scale == 1.0 / cmax
    assert abs(res.iters - ora.iters) <= 1
    assert abs(res.objective - ora.objective) <= 1e-5 * abs(ora.objective)


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_dense_cost_is_rejected(bad):
    n, m = 300, 257
    C = _raw_dense(5, n, m, 1.0)
    C[173, 211] = bad
    dp = _dense_problem(C, np.full(n, 1.0 / n), np.full(m, 1.2 / m), 0.8)
    with pytest.raises(pkg.PotError) as e:
        pkg.aspot_solve(dp, 0.05, 1e-3, max_iter=100)
    assert e.value.status == 1 and "NaN/Inf" in str(e.value)
    with pytest.raises(pkg.PotError) as e:
        pkg.pot_cost_max(dp)
    assert e.value.status == 1


def test_nan_coordinate_is_rejected_on_both_point_paths():
    # BF16 d = 128 (tcgen05 max-cost pass)
    pb = W.cloud_32k(4, n=300, m=260)
    pb.X_bf16 = pb.X_bf16.copy()
    pb.X_bf16[77, 5] = 0x7FC0                       # BF16 quiet NaN
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    with pytest.raises(pkg.PotError) as e:
        pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=50)
    assert e.value.status == 1
    # FP32 d = 3 (CUDA-core pass with register-resident coordinates)
    g = np.random.default_rng(2)
    X = torch.tensor(g.uniform(0, 1, (200, 3)), dtype=torch.float32, device="cuda")
    Y = torch.tensor(g.uniform(0, 1, (150, 3)), dtype=torch.float32, device="cuda")
    Y[42, 1] = float("nan")
    dp = pkg.DeviceProblem(pkg.COST_SQEUCLID_F32, _t(np.full(200, 1 / 200)), _t(np.full(150, 1.2 / 150)), 0.8,
                           X=X, Y=Y, cost_scale=0.0)
    with pytest.raises(pkg.PotError) as e:
        pkg.aspot_solve(dp, 0.05, 1e-3, max_iter=50)
    assert e.value.status == 1
