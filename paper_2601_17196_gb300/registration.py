"""ctypes binding of ``include/registration.h`` and the host loop of batched
rigid point-cloud registration through POT (appendix, "Point Cloud
Registration"): for every pair still moving, one batched ASPOT solve on the
current source, the weighted Procrustes fit of the rounded plan and the motion
applied to the source, all in the library's kernels; this module keeps the
list of pairs that have not converged and the annealed gamma."""
from __future__ import annotations

import ctypes as ct
import dataclasses
from typing import List, Sequence

import numpy as np
import torch

from . import binding as B


def _ptr_array(tensors) -> ct.Array:
    return (ct.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])


def _ws(count: int, device) -> torch.Tensor:
    b = ct.c_size_t(0)
    B._check(B.lib().pot_rigid_workspace_size(int(count), ct.byref(b)))
    buf = torch.empty(int(b.value) + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + int(b.value)]


def rigid_fit(probs: Sequence[B.DeviceProblem], plans: Sequence[B.Plan], gamma: float,
              y0: Sequence[torch.Tensor]) -> torch.Tensor:
    """[count, 16] FP64 on the device: R (row-major 9), t (3), |pi|_1, det sign, sweeps, 0."""
    count = len(probs)
    fit = torch.empty(count, 16, dtype=torch.float64, device=probs[0].r.device)
    parr = (B._Problem * count)(*[p.struct() for p in probs])
    plarr = (B._Plan * count)(*[pl.struct() for pl in plans])
    ws = _ws(count, fit.device)
    side, cur = B._stream()
    B._check(B.lib().pot_rigid_fit(parr, count, plarr, float(gamma), ct.cast(_ptr_array(y0), ct.c_void_p),
                                   ct.c_void_p(fit.data_ptr()), ct.c_void_p(ws.data_ptr()), ws.numel(),
                                   ct.c_void_p(side.cuda_stream)))
    side.synchronize()
    B._finish(side, cur)
    return fit


def rigid_apply(probs: Sequence[B.DeviceProblem], y0: Sequence[torch.Tensor], fit: torch.Tensor) -> None:
    """probs[k].Y <- R_k y0_k + t_k."""
    count = len(probs)
    parr = (B._Problem * count)(*[p.struct() for p in probs])
    ws = _ws(count, fit.device)
    side, cur = B._stream()
    B._check(B.lib().pot_rigid_apply(parr, count, ct.cast(_ptr_array(y0), ct.c_void_p),
                                     ct.c_void_p(fit.data_ptr()), ct.c_void_p(ws.data_ptr()), ws.numel(),
                                     ct.c_void_p(side.cuda_stream)))
    side.synchronize()
    B._finish(side, cur)


@dataclasses.dataclass
class Registration:
    R: np.ndarray
    t: np.ndarray
    registrations: int
    inner_iterations: int
    converged: bool


def register_batched(pairs: Sequence[tuple], alpha: float = 0.4, gamma0: float = 0.02, anneal: float = 0.83,
                     gamma_min: float = 0.002, eps: float = 1e-3, max_reg: int = 60, tol: float = 1e-6,
                     max_iter: int = 20000, device="cuda", autotune: bool = False) -> List[Registration]:
    """Register every (target X [n,3], source Y0 [m,3]) pair: uniform masses
    1/n and 1/m, s = alpha min(n,m)/max(n,m), cost |x - (R y + t)|^2
    (cost_scale 1), gamma_k = max(gamma_min, gamma0 anneal^k); a pair stops
    when |R_k - R_{k-1}|_F + |t_k - t_{k-1}| < tol.  ``autotune`` lets the
    batched solver pick its tile shape (timed once per set of active pairs,
    which changes as pairs finish, then cached); the default tiles already
    suit these 1024-point pairs, so it is off by default."""
    probs, y0s = [], []
    for X, Y0 in pairs:
        n, m = X.shape[0], Y0.shape[0]
        Xd = torch.tensor(np.asarray(X, dtype=np.float32), device=device).contiguous()
        Y0d = torch.tensor(np.asarray(Y0, dtype=np.float32), device=device).contiguous()
        r = torch.full((n,), 1.0 / n, dtype=torch.float64, device=device)
        c = torch.full((m,), 1.0 / m, dtype=torch.float64, device=device)
        s = alpha * min(n, m) / max(n, m)
        probs.append(B.DeviceProblem(B.COST_SQEUCLID_F32, r, c, s, X=Xd, Y=Y0d.clone(), cost_scale=1.0))
        y0s.append(Y0d)
    K = len(pairs)
    Rs = [np.eye(3) for _ in range(K)]
    ts = [np.zeros(3) for _ in range(K)]
    regs = [0] * K
    inner = [0] * K
    done = [False] * K
    for k in range(max_reg):
        active = [i for i in range(K) if not done[i]]
        if not active:
            break
        gam = max(gamma_min, gamma0 * anneal ** k)
        sub = [probs[i] for i in active]
        res = B.aspot_solve_batched(sub, gam, eps, max_iter=max_iter, flags=B.FLAG_AUTOTUNE if autotune else 0)
        fit = rigid_fit(sub, [r.plan for r in res], gam, [y0s[i] for i in active])
        rigid_apply(sub, [y0s[i] for i in active], fit)
        F = fit.cpu().numpy()
        for a, i in enumerate(active):
            R = F[a, :9].reshape(3, 3)
            t = F[a, 9:12].copy()
            delta = np.linalg.norm(R - Rs[i]) + np.linalg.norm(t - ts[i])
            Rs[i], ts[i] = R, t
            regs[i] += 1
            inner[i] += res[a].iters
            if delta < tol:
                done[i] = True
    return [Registration(Rs[i], ts[i], regs[i], inner[i], done[i]) for i in range(K)]
