"""GPU parity of the registration steps (include/registration.h): the
weighted Procrustes fit of an implicit plan and the motion applied to the
source, against the FP64 oracle; and the batched registration loop, which
must recover the motion a partial cloud was moved by, as the oracle's loop
does."""
import numpy as np
import pytest
import torch

import pot_workloads as W
from oracle import pot as O
from oracle import registration as RG
from paper_2601_17196_gb300 import binding as B
from paper_2601_17196_gb300 import registration as PR

pytestmark = pytest.mark.gpu


def _inst(n, m, seed):
    g = np.random.default_rng(seed)
    X = g.uniform(0, 1, size=(n, 3)).astype(np.float32).astype(np.float64)
    Y0 = g.uniform(0, 1, size=(m, 3)).astype(np.float32).astype(np.float64)
    Rm = RG.rotation(g.normal(size=3), g.uniform(0, 0.5))
    tm = g.normal(scale=0.05, size=3)
    Ycur = RG.transform(Y0, Rm, tm).astype(np.float32).astype(np.float64)
    return X, Y0, Ycur


@pytest.mark.parametrize("gamma", [0.05, 0.01])
def test_rigid_fit_matches_oracle(gamma):
    sizes = [(100, 50), (257, 130), (64, 600), (1, 7)]
    probs, plans, y0s, refs = [], [], [], []
    for k, (n, m) in enumerate(sizes):
        X, Y0, Ycur = _inst(n, m, k)
        f, gg, p, q, kap = W.plan_params(n, m, seed=10 + k)
        dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
        pr = B.DeviceProblem(B.COST_SQEUCLID_F32, dev(np.full(n, 1.0 / n)), dev(np.full(m, 1.0 / m)), 0.5,
                             X=torch.tensor(X, dtype=torch.float32, device="cuda"),
                             Y=torch.tensor(Ycur, dtype=torch.float32, device="cuda"), cost_scale=1.0)
        pl = B.Plan.empty(n, m)
        pl.f.copy_(dev(f)); pl.g.copy_(dev(gg)); pl.p.copy_(dev(p)); pl.q.copy_(dev(q)); pl.kappa.fill_(kap)
        probs.append(pr); plans.append(pl); y0s.append(torch.tensor(Y0, dtype=torch.float32, device="cuda"))
        C = O.sqeuclid_cost(X, Ycur, 1.0)
        P = RG.implicit_plan(C, gamma, f, gg, p, q, kap)
        refs.append(RG.rigid_fit(X, Y0, P) if n > 2 else (None, None, float(P.sum())))
    fit = PR.rigid_fit(probs, plans, gamma, y0s).cpu().numpy()
    for k, (R, t, mass) in enumerate(refs):
        assert abs(fit[k, 12] - mass) <= 1e-5 * mass
        Rg = fit[k, :9].reshape(3, 3)
        np.testing.assert_allclose(Rg @ Rg.T, np.eye(3), atol=1e-12)     # a rotation even when degenerate
        assert np.linalg.det(Rg) == pytest.approx(1.0)
        if R is None:
            continue
        np.testing.assert_allclose(Rg, R, atol=2e-5)
        np.testing.assert_allclose(fit[k, 9:12], t, atol=2e-5)


def test_rigid_apply_matches_formula():
    X, Y0, _ = _inst(10, 300, 3)
    Y0d = torch.tensor(Y0, dtype=torch.float32, device="cuda")
    pr = B.DeviceProblem(B.COST_SQEUCLID_F32, torch.full((10,), 0.1, dtype=torch.float64, device="cuda"),
                         torch.full((300,), 1 / 300, dtype=torch.float64, device="cuda"), 0.5,
                         X=torch.tensor(X, dtype=torch.float32, device="cuda"), Y=Y0d.clone(), cost_scale=1.0)
    R = RG.rotation([1, 2, 3], 0.3)
    t = np.array([0.1, -0.2, 0.05])
    fit = torch.zeros(1, 16, dtype=torch.float64, device="cuda")
    fit[0, :9] = torch.tensor(R.reshape(-1))
    fit[0, 9:12] = torch.tensor(t)
    PR.rigid_apply([pr], [Y0d], fit)
    np.testing.assert_allclose(pr.Y.cpu().numpy(), RG.transform(Y0, R, t), atol=2e-7)


def test_batched_registration_recovers_the_motion():
    """Eight misaligned partial clouds (half of a 3-ellipsoid target, rotated
    by up to 0.25 rad and shifted by up to 0.08; seeds 0-7) registered at once
    with alpha = 0.6.  Each must map back onto the target points it was cut
    from to 0.06 (the entropic blur), or else end where the FP64 oracle's own
    loop ends: on seed 3 the oracle stops at 0.062 and on seed 6, a
    near-symmetric shape, its loop slides to another match (0.26), so there
    the synthetic shape limits the result, not the GPU.  (With alpha = 0.4 the
    partial matching lets most sources slide; a recorded finding.)"""
    seeds = list(range(8))
    pairs, truth = [], []
    for seed in seeds:
        X, Y0, Rt, tt = W.registration_3d(seed, n=256, frac=0.5, max_angle=0.25, max_shift=0.08)
        pairs.append((X, Y0))
        truth.append((Rt, tt))
    out = PR.register_batched(pairs, alpha=0.6, gamma0=0.02, anneal=0.83, gamma_min=0.002, eps=1e-3, max_reg=30)
    recovered = 0
    for seed, (X, Y0), (Rt, tt), r in zip(seeds, pairs, truth, out):
        err = max(np.abs(r.R - Rt).max(), np.abs(r.t - tt).max())
        if err < 6e-2:
            recovered += 1
            continue
        s = 0.6 * min(X.shape[0], Y0.shape[0]) / max(X.shape[0], Y0.shape[0])
        Ro, to, _, _ = RG.register(X, Y0, s, gamma0=0.02, anneal=0.83, gamma_min=0.002, eps=1e-3, max_reg=30,
                                   tol=1e-6)
        err_o = max(np.abs(Ro - Rt).max(), np.abs(to - tt).max())
        assert err_o >= 5e-2, (seed, err, err_o)                  # the oracle does not recover it either
        assert max(np.abs(r.R - Ro).max(), np.abs(r.t - to).max()) < 2e-2, (seed, err, err_o)
    assert recovered >= 6
    # the small pair of the oracle test, on both sides
    X, Y0, Rt, tt = W.registration_3d(0, n=120, frac=0.5, max_angle=0.4, max_shift=0.08)
    s = 0.6 * min(60, 120) / 120
    Ro, to, ko, _ = RG.register(X, Y0, s, gamma0=0.02, anneal=0.83, gamma_min=0.002, eps=1e-3, max_reg=30,
                                tol=1e-6)
    g = PR.register_batched([(X, Y0)], alpha=0.6, gamma0=0.02, anneal=0.83, gamma_min=0.002, eps=1e-3,
                            max_reg=30)[0]
    assert np.abs(g.R - Ro).max() < 1e-3 and np.abs(g.t - to).max() < 1e-3
