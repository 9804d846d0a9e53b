"""ctypes binding of ``include/warmstart.h`` (argument marshalling) and the
host loops of the learned warm start: building a training set from ASPOT's
own converged duals, training with Adam, and warm-started solves.  Every
arithmetic step runs in the library's kernels; this module only moves
pointers, shuffles indices and reads back losses.
"""
from __future__ import annotations

import ctypes as ct
import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import binding as B

HIDDEN = 128
EXTRA = 5          # features per point besides the coordinates
MODE_FP32 = 0
MODE_BF16 = 1


def _aligned(nbytes: int, device) -> torch.Tensor:
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + nbytes]


def param_count(d: int) -> int:
    n = ct.c_int64(0)
    B._check(B.lib().pot_ws_param_count(int(d), ct.byref(n)))
    return int(n.value)


def offsets(d: int) -> dict:
    """Start of each parameter block in the flat parameter vector."""
    F, H = d + EXTRA, HIDDEN
    o = {"W1": 0}
    o["b1"] = o["W1"] + H * F
    o["W2"] = o["b1"] + H
    o["U"] = o["W2"] + H * H
    o["b2"] = o["U"] + H * (H + 2)
    o["w3"] = o["b2"] + H
    o["b3"] = o["w3"] + H
    o["total"] = o["b3"] + 1
    return o


@dataclasses.dataclass
class FeatureSet:
    """Instances in feature form: ``feats`` [N][d+5], ``extra`` [K][2] and
    ``target`` [N] on the device, ``off`` (K+1 point offsets) on the host."""
    d: int
    feats: torch.Tensor
    extra: torch.Tensor
    off: np.ndarray
    target: Optional[torch.Tensor] = None
    n_rows: Optional[np.ndarray] = None
    weight: Optional[torch.Tensor] = None

    @property
    def count(self) -> int:
        return int(self.off.shape[0] - 1)

    def struct(self) -> B._WsSet:
        s = B._WsSet()
        s.count, s.d = self.count, self.d
        s.off = self.off.ctypes.data_as(ct.c_void_p)
        s.feats, s.extra = self.feats.data_ptr(), self.extra.data_ptr()
        s.target = None if self.target is None else self.target.data_ptr()
        s.weight = None if self.weight is None else self.weight.data_ptr()
        return s

    def subset(self, idx: Sequence[int]) -> "FeatureSet":
        idx = np.asarray(idx, dtype=np.int64)
        parts, tparts, off = [], [], [0]
        for k in idx:
            a, b = int(self.off[k]), int(self.off[k + 1])
            parts.append(self.feats[a:b])
            if self.target is not None:
                tparts.append(self.target[a:b])
            off.append(off[-1] + b - a)
        wparts = [self.weight[int(self.off[k]):int(self.off[k + 1])] for k in idx] if self.weight is not None else []
        return FeatureSet(self.d, torch.cat(parts).contiguous(), self.extra[torch.as_tensor(idx, device=self.extra.device)].contiguous(),
                          np.asarray(off, dtype=np.int64),
                          torch.cat(tparts).contiguous() if tparts else None,
                          None if self.n_rows is None else self.n_rows[idx],
                          torch.cat(wparts).contiguous() if wparts else None)


def features(probs: Sequence[B.DeviceProblem], gamma: float) -> FeatureSet:
    """pot_ws_features for each problem, into one set (rows then columns)."""
    L = B.lib()
    d = probs[0].d
    sizes = [p.n + p.m for p in probs]
    off = np.zeros(len(probs) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    dev = probs[0].r.device
    feats = torch.empty(int(off[-1]), d + EXTRA, dtype=torch.float32, device=dev)
    extra = torch.empty(len(probs), 2, dtype=torch.float32, device=dev)
    ws = None
    side, cur = B._stream()
    for k, p in enumerate(probs):
        if p.d != d:
            raise ValueError("all problems of a set need the same d")
        b = ct.c_size_t(0)
        B._check(L.pot_ws_features_workspace_size(ct.byref(p.struct()), ct.byref(b)))
        if ws is None or ws.numel() < b.value:
            ws = _aligned(int(b.value), dev)
        B._check(L.pot_ws_features(ct.byref(p.struct()), float(gamma), ct.c_void_p(ws.data_ptr()), ws.numel(),
                                   ct.c_void_p(feats[off[k]:].data_ptr()), ct.c_void_p(extra[k:].data_ptr()),
                                   ct.c_void_p(side.cuda_stream)))
    B._finish(side, cur)
    return FeatureSet(d, feats, extra, off, None, np.asarray([p.n for p in probs], dtype=np.int64))


def targets_into(fs: FeatureSet, k: int, prob: B.DeviceProblem, gamma: float, u: torch.Tensor,
                 v: torch.Tensor, w: float, ws: Optional[torch.Tensor] = None) -> None:
    """target[off[k]:off[k+1]] and the loss weights from the converged duals (pot_ws_targets)."""
    if fs.target is None:
        fs.target = torch.zeros(int(fs.off[-1]), dtype=torch.float32, device=fs.feats.device)
    if fs.weight is None:
        fs.weight = torch.ones(int(fs.off[-1]), dtype=torch.float32, device=fs.feats.device)
    L = B.lib()
    if ws is None:
        b = ct.c_size_t(0)
        B._check(L.pot_ws_features_workspace_size(ct.byref(prob.struct()), ct.byref(b)))
        ws = _aligned(int(b.value), fs.feats.device)
    side, cur = B._stream()
    B._check(L.pot_ws_targets(ct.byref(prob.struct()), float(gamma), ct.c_void_p(u.data_ptr()),
                              ct.c_void_p(v.data_ptr()), float(w), ct.c_void_p(fs.target[int(fs.off[k]):].data_ptr()),
                              ct.c_void_p(fs.weight[int(fs.off[k]):].data_ptr()), ct.c_void_p(ws.data_ptr()),
                              ws.numel(), ct.c_void_p(side.cuda_stream)))
    B._finish(side, cur)


def build_training_set(probs: Sequence[B.DeviceProblem], gamma: float, eps: float, batch: int = 512,
                       max_iter: int = 20000, autotune: bool = True) -> tuple:
    """Features of every problem and, as targets, the duals that batched GPU
    ASPOT converges to (pot_ws_targets).  Returns (set, iterations array).
    ``autotune``: the batched solver's tile shape is timed on the first chunk
    of each size signature and cached for the others."""
    fs = features(probs, gamma)
    iters = np.zeros(len(probs), dtype=np.int64)
    L = B.lib()
    ws = None
    for a in range(0, len(probs), batch):
        chunk = list(probs[a:a + batch])
        res = B.aspot_solve_batched(chunk, gamma, eps, max_iter=max_iter, flags=B.FLAG_AUTOTUNE if autotune else 0)
        ws_w = torch.cat([r.plan.w for r in res]).cpu().numpy()
        for j, r in enumerate(res):
            iters[a + j] = r.iters
            b = ct.c_size_t(0)
            B._check(L.pot_ws_features_workspace_size(ct.byref(chunk[j].struct()), ct.byref(b)))
            if ws is None or ws.numel() < b.value:
                ws = _aligned(int(b.value), fs.feats.device)
            targets_into(fs, a + j, chunk[j], gamma, r.plan.u, r.plan.v, float(ws_w[j]), ws)
    return fs, iters


class WarmStartNet:
    """Parameters (flat FP32 device vector, layout of include/warmstart.h) and
    Adam state of the warm-start network."""

    def __init__(self, d: int = 2, seed: int = 0, mode: int = MODE_FP32, device="cuda",
                 params: Optional[torch.Tensor] = None):
        self.d, self.mode, self.device = int(d), int(mode), torch.device(device)
        self.P = param_count(d)
        if params is None:
            self.params = torch.empty(self.P, dtype=torch.float32, device=self.device)
            side, cur = B._stream()
            B._check(B.lib().pot_ws_init(ct.c_void_p(self.params.data_ptr()), self.d, ct.c_uint64(seed),
                                         ct.c_void_p(side.cuda_stream)))
            B._finish(side, cur)
        else:
            if params.numel() != self.P:
                raise ValueError(f"expected {self.P} parameters, got {params.numel()}")
            self.params = params.to(self.device, torch.float32).contiguous().clone()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._ws = None

    # -------------------------------------------------------- plumbing
    def _workspace(self, fs: FeatureSet, nb: int):
        b = ct.c_size_t(0)
        s = fs.struct()
        B._check(B.lib().pot_ws_workspace_size(ct.byref(s), int(nb), ct.byref(b)))
        need = int(b.value)
        if self._ws is None or self._ws.numel() < need:
            self._ws = _aligned(need, self.device)
        return self._ws, self._ws.numel()

    @staticmethod
    def _idx(idx) -> np.ndarray:
        return np.ascontiguousarray(np.asarray(idx, dtype=np.int32))

    # ------------------------------------------------------- operations
    def forward(self, fs: FeatureSet, idx: Sequence[int]) -> torch.Tensor:
        ix = self._idx(idx)
        n = int(sum(int(fs.off[k + 1] - fs.off[k]) for k in ix))
        y = torch.empty(n, dtype=torch.float32, device=self.device)
        ws, nbytes = self._workspace(fs, len(ix))
        side, cur = B._stream()
        B._check(B.lib().pot_ws_forward(ct.byref(fs.struct()), ix.ctypes.data_as(ct.c_void_p), len(ix),
                                        ct.c_void_p(self.params.data_ptr()), self.mode, ct.c_void_p(y.data_ptr()),
                                        ct.c_void_p(ws.data_ptr()), nbytes, ct.c_void_p(side.cuda_stream)))
        B._finish(side, cur)
        return y

    def gradient(self, fs: FeatureSet, idx: Sequence[int]):
        ix = self._idx(idx)
        g = torch.empty(self.P, dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        ws, nbytes = self._workspace(fs, len(ix))
        side, cur = B._stream()
        B._check(B.lib().pot_ws_gradient(ct.byref(fs.struct()), ix.ctypes.data_as(ct.c_void_p), len(ix),
                                         ct.c_void_p(self.params.data_ptr()), self.mode, ct.c_void_p(g.data_ptr()),
                                         ct.c_void_p(loss.data_ptr()), ct.c_void_p(ws.data_ptr()), nbytes,
                                         ct.c_void_p(side.cuda_stream)))
        B._finish(side, cur)
        return g, loss

    def train_step(self, fs: FeatureSet, idx: Sequence[int], lr: float = 1e-3, beta1: float = 0.9,
                   beta2: float = 0.999, eps: float = 1e-8) -> torch.Tensor:
        ix = self._idx(idx)
        self.step += 1
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        opt = B._WsAdam(float(lr), float(beta1), float(beta2), float(eps))
        ws, nbytes = self._workspace(fs, len(ix))
        side, cur = B._stream()
        B._check(B.lib().pot_ws_train_step(ct.byref(fs.struct()), ix.ctypes.data_as(ct.c_void_p), len(ix),
                                           ct.c_void_p(self.params.data_ptr()), ct.c_void_p(self.m.data_ptr()),
                                           ct.c_void_p(self.v.data_ptr()), ct.byref(opt), self.step, self.mode,
                                           ct.c_void_p(loss.data_ptr()), ct.c_void_p(ws.data_ptr()), nbytes,
                                           ct.c_void_p(side.cuda_stream)))
        B._finish(side, cur)
        return loss

    def fit(self, fs: FeatureSet, epochs: int, batch: int = 32, lr: float = 1e-3, lr_final: float = 1e-4,
            seed: int = 0) -> List[float]:
        """Adam over shuffled mini-batches of instances; the learning rate
        decays geometrically from lr to lr_final.  Returns the mean batch loss
        of every epoch."""
        rng = np.random.default_rng(seed)
        K = fs.count
        steps = max(1, epochs * ((K + batch - 1) // batch))
        decay = (lr_final / lr) ** (1.0 / steps) if steps > 1 else 1.0
        cur = lr
        hist = []
        for _ in range(epochs):
            perm = rng.permutation(K)
            losses = []
            for a in range(0, K, batch):
                losses.append(self.train_step(fs, perm[a:a + batch], lr=cur))
                cur *= decay
            hist.append(float(torch.cat(losses).mean().item()))
        return hist

    def warm_start(self, prob: B.DeviceProblem, gamma: float):
        """(u0, v0, w0) for aspot_solve: u0 = log r - softplus(y / gamma),
        v0 likewise, then the shift step (pot_ws_warm_start)."""
        L = B.lib()
        b = ct.c_size_t(0)
        B._check(L.pot_ws_warm_workspace_size(ct.byref(prob.struct()), ct.byref(b)))
        need = int(b.value)
        if self._ws is None or self._ws.numel() < need:
            self._ws = _aligned(need, self.device)
        u0 = torch.empty(prob.n, dtype=torch.float64, device=self.device)
        v0 = torch.empty(prob.m, dtype=torch.float64, device=self.device)
        w0 = ct.c_double(0.0)
        side, cur = B._stream()
        B._check(L.pot_ws_warm_start(ct.byref(prob.struct()), float(gamma), ct.c_void_p(self.params.data_ptr()),
                                     self.d, self.mode, ct.c_void_p(u0.data_ptr()), ct.c_void_p(v0.data_ptr()),
                                     ct.byref(w0), ct.c_void_p(self._ws.data_ptr()), self._ws.numel(),
                                     ct.c_void_p(side.cuda_stream)))
        B._finish(side, cur)
        return u0, v0, float(w0.value)

    def solve(self, prob: B.DeviceProblem, gamma: float, eps: float, max_iter: int = 20000, flags: int = 0,
              block_rule: int = B.BLOCK_CYCLIC):
        """Warm-started ASPOT with the zero-start fallback (POT_FLAG_WARM_CHECK)."""
        u0, v0, w0 = self.warm_start(prob, gamma)
        return B.aspot_solve(prob, gamma, eps, max_iter=max_iter, flags=flags | B.FLAG_WARM_CHECK,
                             u0=u0, v0=v0, w0=w0, block_rule=block_rule)

    def state(self) -> dict:
        return {"d": self.d, "params": self.params.detach().cpu().numpy().copy(), "step": self.step}
