"""GPU parity of the learned warm start (include/warmstart.h): features,
forward pass, gradients and one Adam step against the FP64 oracle of the
network; the E(z_warm) > E(0) fallback of aspot_solve; and what a trained
network gains over the zero start."""
import numpy as np
import pytest
import torch

import pot_workloads as W
from oracle import pot as O
from oracle import warmstart as OW
from paper_2601_17196_gb300 import binding as B
from paper_2601_17196_gb300 import warmstart as WS

pytestmark = pytest.mark.gpu


def _set(sizes, d, seed):
    feats, extra, target, off = W.ws_batch(sizes, d, seed)
    fs = WS.FeatureSet(d, torch.from_numpy(feats).cuda(), torch.from_numpy(extra).cuda(), off,
                       torch.from_numpy(target).cuda())
    return fs, feats, extra, target, off


def _oracle(P, feats, extra, target, off, idx, weight=None):
    fe = np.vstack([feats[off[k]:off[k + 1]] for k in idx]).astype(np.float64)
    tg = np.concatenate([target[off[k]:off[k + 1]] for k in idx]).astype(np.float64)
    wt = None if weight is None else np.concatenate([weight[off[k]:off[k + 1]] for k in idx]).astype(np.float64)
    seg = np.concatenate([np.full(off[k + 1] - off[k], b) for b, k in enumerate(idx)])
    ex = extra[idx].astype(np.float64)
    y, cache = OW.forward(P, fe, seg, ex)
    g = OW.backward(P, fe, seg, ex, tg, cache, wt)
    return y, OW.mse(y, tg, wt), g


# ragged tiles (300 = 2 x 128 + 44), a one-point instance, exactly one tile
SIZES = [300, 77, 129, 128, 1, 513]


# tolerances: FP32 mode 1e-4 of each gradient block's largest entry; BF16
# mode (8-bit mantissa operands: relative rounding 2^-9 per factor, summed
# over 128-term products) 2e-2
TOL = {WS.MODE_FP32: (2e-5, 1e-4, 1e-4), WS.MODE_BF16: (1e-2, 2e-2, 2e-2)}


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("mode", [WS.MODE_FP32, WS.MODE_BF16])
@pytest.mark.parametrize("d", [2, 3])
def test_forward_and_gradient_match_oracle(d, mode, weighted):
    fs, feats, extra, target, off = _set(SIZES, d, 1)
    wts = W.ws_weights(int(off[-1]), 7) if weighted else None
    if weighted:
        fs.weight = torch.from_numpy(wts).cuda()
    flat = W.ws_params(d, 2)
    net = WS.WarmStartNet(d, params=torch.from_numpy(flat), mode=mode)
    idx = [2, 0, 4, 5, 1]                     # a shuffled subset
    y = net.forward(fs, idx).cpu().numpy().astype(np.float64)
    g, loss = net.gradient(fs, idx)
    P = OW.unflatten(flat.astype(np.float64), d)
    yo, lo, go = _oracle(P, feats, extra, target, off, idx, wts)
    ty, tl, tg = TOL[mode]
    assert np.abs(y - yo).max() <= ty * max(1.0, np.abs(yo).max())
    assert abs(loss.item() - lo) <= tl * lo
    G = OW.unflatten(g.cpu().numpy().astype(np.float64), d)
    tgt = np.concatenate([target[off[k]:off[k + 1]] for k in idx]).astype(np.float64)
    for k in OW.ORDER:
        err, ref = np.abs(G[k] - go[k]).max(), _scale(go, k, yo, tgt)
        assert err <= tg * ref + 1e-10, (k, err, ref)


def _scale(go, k, y, t):
    """Size of a gradient block's terms: its largest entry, except for db3 =
    (2/N) sum w (y - t), whose terms cancel; its scale is (2/N) sum |y - t|."""
    if k == "b3":
        return 2.0 * np.abs(y - t).mean()
    return np.abs(go[k]).max()


def test_bf16_many_tiles_per_cta():
    """More tiles than SMs: each persistent CTA accumulates several tiles in TMEM."""
    d = 2
    sizes = [200 + 37 * k for k in range(60)]          # 60 instances, ~230 tiles
    fs, feats, extra, target, off = _set(sizes, d, 9)
    flat = W.ws_params(d, 10)
    idx = list(range(60))
    g32, l32 = WS.WarmStartNet(d, params=torch.from_numpy(flat), mode=WS.MODE_FP32).gradient(fs, idx)
    g16, l16 = WS.WarmStartNet(d, params=torch.from_numpy(flat), mode=WS.MODE_BF16).gradient(fs, idx)
    G32 = OW.unflatten(g32.cpu().numpy().astype(np.float64), d)
    G16 = OW.unflatten(g16.cpu().numpy().astype(np.float64), d)
    assert abs(l16.item() - l32.item()) <= 2e-2 * l32.item()
    y32 = WS.WarmStartNet(d, params=torch.from_numpy(flat)).forward(fs, idx).cpu().numpy().astype(np.float64)
    for k in OW.ORDER:
        err, ref = np.abs(G16[k] - G32[k]).max(), _scale(G32, k, y32, target.astype(np.float64))
        assert err <= 2e-2 * ref + 1e-10, (k, err, ref)


def test_gradient_is_deterministic_and_batch_order_free():
    d = 2
    fs, *_ = _set(SIZES, d, 3)
    net = WS.WarmStartNet(d, params=torch.from_numpy(W.ws_params(d, 4)))
    g1, l1 = net.gradient(fs, [0, 1, 2, 3])
    g2, l2 = net.gradient(fs, [0, 1, 2, 3])
    assert torch.equal(g1, g2) and torch.equal(l1, l2)
    g3, _ = net.gradient(fs, [3, 1, 0, 2])
    assert torch.allclose(g1, g3, rtol=1e-5, atol=1e-7 * g1.abs().max().item())


def test_adam_step_matches_oracle():
    d = 2
    fs, feats, extra, target, off = _set(SIZES, d, 5)
    flat = W.ws_params(d, 6)
    net = WS.WarmStartNet(d, params=torch.from_numpy(flat))
    idx = [0, 1, 2, 3, 4, 5]
    lr = 1e-3
    loss = net.train_step(fs, idx, lr=lr)
    P = OW.unflatten(flat.astype(np.float64), d)
    _, lo, go = _oracle(P, feats, extra, target, off, idx)
    assert abs(loss.item() - lo) <= 1e-4 * lo
    M = {k: np.zeros_like(v) for k, v in P.items()}
    V = {k: np.zeros_like(v) for k, v in P.items()}
    OW.adam_step(P, go, M, V, step=1, lr=lr)
    Q = OW.unflatten(net.params.cpu().numpy().astype(np.float64), d)
    for k in OW.ORDER:
        # the first step is lr * g / (|g| + eps): exact where |g| is well above
        # the FP32 gradient error, at most 2 lr apart where g is near zero
        big = np.abs(go[k]) > 1e-2 * np.abs(go[k]).max()
        assert np.abs(Q[k] - P[k])[big].max() <= 2e-6, k
        assert np.abs(Q[k] - P[k]).max() <= 2 * lr + 1e-6, k


@pytest.mark.parametrize("kind", [B.COST_SQEUCLID_F32, B.COST_SQEUCLID_BF16])
def test_features_match_oracle(kind):
    pb = W.mix_2d(3, n=300, m=200)
    if kind == B.COST_SQEUCLID_BF16:
        pb.X_bf16, pb.Y_bf16 = W.to_bf16_bits(pb.X), W.to_bf16_bits(pb.Y)
        X, Y = W.from_bf16_bits(pb.X_bf16), W.from_bf16_bits(pb.Y_bf16)
    else:
        X, Y = pb.X, pb.Y
    dp = B.DeviceProblem.from_workload(pb, kind=kind)
    fs = WS.features([dp], pb.gamma)
    f = fs.feats.cpu().numpy().astype(np.float64)
    e = fs.extra.cpu().numpy().astype(np.float64)[0]
    fo, eo = OW.features(X, Y, pb.r, pb.c, pb.s, pb.gamma, pb.cost_scale)
    assert f.shape == fo.shape
    assert np.abs(f - fo).max() <= 1e-5 * max(1.0, np.abs(fo).max())
    np.testing.assert_allclose(e, eo, rtol=1e-6)


def test_warm_check_keeps_zero_start_when_the_start_is_worse():
    pb = W.mix_2d(5, n=256)
    dp = B.DeviceProblem.from_workload(pb, kind=B.COST_SQEUCLID_F32)
    cold = B.aspot_solve(dp, pb.gamma, pb.eps)
    assert cold.status == 0
    u0 = torch.full((dp.n,), 3.0, dtype=torch.float64, device="cuda")
    v0 = torch.full((dp.m,), 3.0, dtype=torch.float64, device="cuda")
    r = B.aspot_solve(dp, pb.gamma, pb.eps, flags=B.FLAG_WARM_CHECK, u0=u0, v0=v0, w0=0.0)
    assert r.warm_used == 0 and r.err_warm > r.err_zero
    assert r.iters == cold.iters and r.objective == cold.objective
    # both residuals against the oracle's E at the same points (Algorithm 2's setup)
    C = O.sqeuclid_cost(pb.X, pb.Y, pb.cost_scale)
    st = O.approx_setup(pb.r, pb.c, pb.s, pb.eps, float(C.max()), pb.gamma)
    ew = O.feas_error(C, st.gamma, st.r_t, st.c_t, pb.s, O.Dual(np.full(dp.n, 3.0), np.full(dp.m, 3.0), 0.0))
    ez = O.feas_error(C, st.gamma, st.r_t, st.c_t, pb.s, O.Dual.zeros(dp.n, dp.m))
    assert abs(r.err_warm - ew) <= 1e-5 * ew
    assert abs(r.err_zero - ez) <= 1e-5 * ez
    # a start at the converged duals is kept and stops at once
    good = B.aspot_solve(dp, pb.gamma, pb.eps, flags=B.FLAG_WARM_CHECK, u0=cold.plan.u.clone(),
                         v0=cold.plan.v.clone(), w0=float(cold.plan.w.item()))
    assert good.warm_used == 1 and good.err_warm < good.err_zero
    assert good.status == 0 and good.iters <= 3
    assert abs(good.objective - cold.objective) <= pb.eps


@pytest.mark.parametrize("mode", [WS.MODE_BF16])
def test_trained_network_cuts_iterations_to_eps(mode):
    """Train on ASPOT's own duals (mixtures of 2-6 Gaussians in 2-D, n = m =
    1024, gamma = 0.02, eps = 1e-3), then solve held-out seeds from the
    network's start and from zero: the warm starts must need fewer
    iterations on average, and both must meet the same accuracy."""
    gamma, eps = 0.02, 1e-3
    train = [B.DeviceProblem.from_workload(W.mix_2d(10_000 + k), kind=B.COST_SQEUCLID_F32) for k in range(1024)]
    fs, iters = WS.build_training_set(train, gamma, eps)
    assert np.all(iters > 0)
    net = WS.WarmStartNet(2, seed=0, mode=mode)
    hist = net.fit(fs, epochs=60, batch=32, lr=3e-3, lr_final=3e-5, seed=0)
    assert hist[-1] < 0.1 * hist[0]
    cold_it, warm_it, used = [], [], []
    for seed in range(32):
        pb = W.mix_2d(seed)
        dp = B.DeviceProblem.from_workload(pb, kind=B.COST_SQEUCLID_F32)
        c = B.aspot_solve(dp, gamma, eps, max_iter=20000)
        w = net.solve(dp, gamma, eps)
        assert c.status == 0 and w.status == 0
        # both are eps-solutions of the same problem
        assert abs(w.objective - c.objective) <= eps
        cold_it.append(c.iters)
        warm_it.append(w.iters)
        used.append(w.warm_used)
    print("cold", np.mean(cold_it), "warm", np.mean(warm_it), "warm used", np.mean(used))
    assert np.mean(warm_it) < 0.9 * np.mean(cold_it)


def test_targets_match_oracle():
    pb = W.mix_2d(7, n=200, m=150)
    dp = B.DeviceProblem.from_workload(pb, kind=B.COST_SQEUCLID_F32)
    g = np.random.default_rng(8)
    u, v, w = g.normal(-8, 2, size=dp.n), g.normal(-8, 2, size=dp.m), 3.0
    fs = WS.FeatureSet(2, torch.zeros(dp.n + dp.m, 7, device="cuda"), torch.zeros(1, 2, device="cuda"),
                       np.array([0, dp.n + dp.m], dtype=np.int64))
    WS.targets_into(fs, 0, dp, 0.02, torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda"), w)
    t = fs.target.cpu().numpy().astype(np.float64)
    C = O.sqeuclid_cost(pb.X, pb.Y, pb.cost_scale)
    to = OW.targets(C, 0.02, u, v, w)
    # FP32 pass log-sums (5e-6 + 2e-7 |lse|) times gamma
    assert np.abs(t - to).max() <= 0.02 * (5e-6 + 2e-7 * np.abs(to / 0.02).max()) + 1e-7
    wo = OW.target_weights(C, 0.02, u, v, w)
    assert np.abs(fs.weight.cpu().numpy() - wo).max() <= 2e-5


@pytest.mark.parametrize("cost_scale", [0.0, 0.7])
def test_warm_start_matches_oracle(cost_scale):
    """pot_ws_warm_start (features, forward, duals, shift step) against the
    oracle's restatement with the same parameters, FP32 mode."""
    pb = W.mix_2d(11, n=160, m=230)
    pb.cost_scale = cost_scale
    dp = B.DeviceProblem.from_workload(pb, kind=B.COST_SQEUCLID_F32)
    flat = W.ws_params(2, 12, bias_scale=0.02)
    net = WS.WarmStartNet(2, params=torch.from_numpy(flat))
    u0, v0, w0 = net.warm_start(dp, pb.gamma)
    uo, vo, wo = OW.warm_start(OW.unflatten(flat.astype(np.float64), 2), pb.X, pb.Y, pb.r, pb.c, pb.s, pb.gamma,
                               cost_scale)
    # FP32 network output divided by gamma: 1e-6 relative of |y| <= 1 becomes ~5e-5 in u
    np.testing.assert_allclose(u0.cpu().numpy(), uo, atol=2e-3)
    np.testing.assert_allclose(v0.cpu().numpy(), vo, atol=2e-3)
    assert abs(w0 - wo) <= 2e-3 * max(1.0, abs(wo))
