"""ctypes binding of ``include/aspot.h``: argument marshalling only.

Every step of the solvers runs inside ``lib/libaspot.so``.  torch provides the
device buffers (workspace, plan vectors) and the stream.
"""
from __future__ import annotations

import ctypes as ct
import dataclasses
import os
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libaspot.so")

FLAG_STOP_RAW_EPS = 1
FLAG_NO_SMOOTH = 2
FLAG_TRACE = 4
FLAG_NO_STOP = 8
FLAG_FORCE_SIMT = 16
FLAG_PROFILE = 32
FLAG_WARM_CHECK = 64
FLAG_AUTOTUNE = 128
FLAG_STAGED = 256

COST_DENSE_F32 = 0
COST_SQEUCLID_BF16 = 1
COST_SQEUCLID_F16 = 2
COST_SQEUCLID_F32 = 3
BLOCK_CYCLIC = 0
BLOCK_GREEDY = 1

STATUS = {0: "POT_OK", 1: "POT_EINVAL", 2: "POT_ENOMEM", 3: "POT_ECUDA", 4: "POT_ENOCONV",
          5: "POT_ENONFINITE", 6: "POT_ETIMEOUT"}

EXPORTED = ["pot_workspace_size", "aspot_solve", "sinkhorn_pot_solve", "pot_round", "pot_objective",
            "pot_marginals", "pot_marginals_workspace_size", "pot_pass_status", "pot_cost_max", "pot_plan_dense", "pot_trace", "aspot_state_export",
            "pot_workspace_size_batched",
            "aspot_solve_batched", "pot_marginals_static", "pot_ws_param_count", "pot_ws_init",
            "pot_ws_features_workspace_size", "pot_ws_features", "pot_ws_targets", "pot_ws_workspace_size", "pot_ws_forward", "pot_ws_gradient",
            "pot_ws_train_step", "pot_ws_warm_workspace_size", "pot_ws_warm_start", "pot_rigid_workspace_size",
            "pot_rigid_fit", "pot_rigid_apply", "pot_trace_batched", "pot_autotune_set", "pot_autotune_lookup",
            "pot_autotune_clear",
            "pot_autotune_save", "pot_autotune_load", "pot_pass_kernel", "pot_last_error"]


class PotError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Problem(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("m", ct.c_int64), ("kind", ct.c_int32),
                ("C", ct.c_void_p), ("ldc", ct.c_int64),
                ("X", ct.c_void_p), ("Y", ct.c_void_p), ("d", ct.c_int32), ("ldx", ct.c_int64), ("ldy", ct.c_int64),
                ("cost_scale", ct.c_double), ("r", ct.c_void_p), ("c", ct.c_void_p), ("s", ct.c_double)]


class _Params(ct.Structure):
    _fields_ = [("gamma", ct.c_double), ("eps", ct.c_double), ("p_tune", ct.c_double),
                ("max_iter", ct.c_int32), ("block_rule", ct.c_int32), ("flags", ct.c_int32),
                ("check_every", ct.c_int32), ("u0", ct.c_void_p), ("v0", ct.c_void_p), ("w0", ct.c_double),
                ("resume", ct.c_void_p), ("wait_limit_ns", ct.c_int64)]


class _State(ct.Structure):
    _fields_ = [("u_tilde", ct.c_void_p), ("v_tilde", ct.c_void_p), ("u_check", ct.c_void_p),
                ("v_check", ct.c_void_p), ("w_tilde", ct.c_double), ("w_check", ct.c_double),
                ("phi_check", ct.c_double), ("theta", ct.c_double), ("t", ct.c_int32), ("pad", ct.c_int32)]


class _WsSet(ct.Structure):
    _fields_ = [("count", ct.c_int64), ("d", ct.c_int32), ("pad", ct.c_int32), ("off", ct.c_void_p),
                ("feats", ct.c_void_p), ("extra", ct.c_void_p), ("target", ct.c_void_p), ("weight", ct.c_void_p)]


class _WsAdam(ct.Structure):
    _fields_ = [("lr", ct.c_float), ("beta1", ct.c_float), ("beta2", ct.c_float), ("eps", ct.c_float)]


class _Plan(ct.Structure):
    _fields_ = [(k, ct.c_void_p) for k in ("u", "v", "w", "f", "g", "p", "q", "kappa")]


class _Result(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("iters", ct.c_int32), ("objective", ct.c_double),
                ("err_final", ct.c_double), ("eps_stop", ct.c_double), ("gamma", ct.c_double),
                ("cost_scale", ct.c_double), ("mass", ct.c_double), ("ms", ct.c_double),
                ("rounding_branch", ct.c_int32), ("nonfinite", ct.c_int32),
                ("pass_ms", ct.c_double), ("pass_launches", ct.c_int64), ("kernel_launches", ct.c_int64),
                ("err_warm", ct.c_double), ("err_zero", ct.c_double), ("warm_used", ct.c_int32),
                ("tile_rows", ct.c_int32), ("tile_cols", ct.c_int32), ("cluster_loop", ct.c_int32),
                ("tune_ms", ct.c_double)]


_lib_handle = None


def lib() -> ct.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = ct.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_double
        P, Q, PL, R = ct.POINTER(_Problem), ct.POINTER(_Params), ct.POINTER(_Plan), ct.POINTER(_Result)
        L.pot_workspace_size.argtypes = [P, Q, ct.POINTER(ct.c_size_t)]
        L.aspot_solve.argtypes = [P, Q, vp, ct.c_size_t, PL, R, vp]
        L.sinkhorn_pot_solve.argtypes = [P, Q, vp, ct.c_size_t, PL, R, vp]
        L.pot_round.argtypes = [P, dbl, vp, vp, dbl, vp, ct.c_size_t, PL, ct.POINTER(i32), vp]
        L.pot_objective.argtypes = [P, PL, dbl, vp, ct.c_size_t, ct.POINTER(dbl), vp]
        L.pot_marginals.argtypes = [P, dbl, vp, vp, dbl, vp, ct.c_size_t, vp, vp, vp, vp]
        L.pot_pass_status.argtypes = [vp, vp]
        L.pot_marginals_workspace_size.argtypes = [P, ct.POINTER(ct.c_size_t)]
        L.pot_cost_max.argtypes = [P, vp, ct.c_size_t, ct.POINTER(dbl), vp]
        L.pot_plan_dense.argtypes = [P, PL, dbl, vp, i64, vp]
        L.pot_trace.argtypes = [vp, i32, vp, vp]
        L.aspot_state_export.argtypes = [P, Q, vp, ct.c_size_t, ct.POINTER(_State), vp]
        L.pot_workspace_size_batched.argtypes = [P, i32, ct.POINTER(ct.c_size_t)]
        L.aspot_solve_batched.argtypes = [P, i32, Q, vp, ct.c_size_t, PL, R, vp]
        L.pot_marginals_static.argtypes = [P, dbl, vp, vp, dbl, vp, vp, vp, vp]
        WS, AD, sz = ct.POINTER(_WsSet), ct.POINTER(_WsAdam), ct.c_size_t
        L.pot_ws_param_count.argtypes = [i32, ct.POINTER(i64)]
        L.pot_ws_init.argtypes = [vp, i32, ct.c_uint64, vp]
        L.pot_ws_features_workspace_size.argtypes = [P, ct.POINTER(sz)]
        L.pot_ws_features.argtypes = [P, dbl, vp, sz, vp, vp, vp]
        L.pot_ws_targets.argtypes = [P, dbl, vp, vp, dbl, vp, vp, vp, sz, vp]
        L.pot_ws_workspace_size.argtypes = [WS, i32, ct.POINTER(sz)]
        L.pot_ws_forward.argtypes = [WS, vp, i32, vp, i32, vp, vp, sz, vp]
        L.pot_ws_gradient.argtypes = [WS, vp, i32, vp, i32, vp, vp, vp, sz, vp]
        L.pot_ws_train_step.argtypes = [WS, vp, i32, vp, vp, vp, AD, i64, i32, vp, vp, sz, vp]
        L.pot_ws_warm_workspace_size.argtypes = [P, ct.POINTER(sz)]
        L.pot_ws_warm_start.argtypes = [P, dbl, vp, i32, i32, vp, vp, ct.POINTER(dbl), vp, sz, vp]
        L.pot_rigid_workspace_size.argtypes = [i32, ct.POINTER(sz)]
        L.pot_rigid_fit.argtypes = [P, i32, PL, dbl, vp, vp, vp, sz, vp]
        L.pot_rigid_apply.argtypes = [P, i32, vp, vp, vp, sz, vp]
        L.pot_trace_batched.argtypes = [vp, P, i32, i32, vp, vp]
        L.pot_autotune_set.argtypes = [P, i32, i32, i32]
        L.pot_autotune_lookup.argtypes = [P, i32, ct.POINTER(i32), ct.POINTER(i32)]
        L.pot_autotune_clear.argtypes = []
        L.pot_autotune_save.argtypes = [ct.c_char_p]
        L.pot_autotune_load.argtypes = [ct.c_char_p]
        L.pot_pass_kernel.argtypes = [P, i32]
        for name in EXPORTED[:-2]:
            getattr(L, name).restype = ct.c_int
        L.pot_pass_kernel.restype = ct.c_char_p
        L.pot_last_error.restype = ct.c_char_p
        _lib_handle = L
    return _lib_handle


def exported_symbols() -> list:
    return list(EXPORTED)


def _check(status: int, allow=(0,)):
    if status not in allow:
        raise PotError(status, lib().pot_last_error().decode())
    return status


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


@dataclasses.dataclass
class DeviceProblem:
    """Device copies of one POT instance (see include/aspot.h)."""
    kind: int
    r: torch.Tensor
    c: torch.Tensor
    s: float
    C: Optional[torch.Tensor] = None
    X: Optional[torch.Tensor] = None
    Y: Optional[torch.Tensor] = None
    cost_scale: float = 0.0

    @property
    def n(self) -> int:
        return int(self.r.shape[0])

    @property
    def m(self) -> int:
        return int(self.c.shape[0])

    @property
    def d(self) -> int:
        return 0 if self.X is None else int(self.X.shape[1])

    def struct(self) -> _Problem:
        p = _Problem()
        p.n, p.m, p.kind = self.n, self.m, self.kind
        if self.C is not None:
            p.C, p.ldc = self.C.data_ptr(), self.C.stride(0)
        if self.X is not None:
            p.X, p.Y, p.d = self.X.data_ptr(), self.Y.data_ptr(), self.d
            p.ldx, p.ldy = self.X.stride(0), self.Y.stride(0)
        p.cost_scale = self.cost_scale
        p.r, p.c, p.s = self.r.data_ptr(), self.c.data_ptr(), float(self.s)
        return p

    @staticmethod
    def from_workload(pb, device="cuda", kind: Optional[int] = None) -> "DeviceProblem":
        """From a ``pot_workloads.Problem``: dense FP32 cost when it has one,
        else BF16 points when it carries BF16 bit patterns, else FP32 points."""
        r = torch.tensor(pb.r, dtype=torch.float64, device=device)
        c = torch.tensor(pb.c, dtype=torch.float64, device=device)
        if kind is None:
            kind = COST_DENSE_F32 if pb.C is not None else (COST_SQEUCLID_BF16 if pb.X_bf16 is not None else COST_SQEUCLID_F32)
        if kind == COST_DENSE_F32:
            C = torch.from_numpy(np.ascontiguousarray(pb.C, dtype=np.float32)).to(device)
            return DeviceProblem(kind, r, c, pb.s, C=C, cost_scale=pb.cost_scale)
        if kind == COST_SQEUCLID_BF16:
            X = torch.from_numpy(pb.X_bf16.view(np.int16)).to(device).view(torch.bfloat16)
            Y = torch.from_numpy(pb.Y_bf16.view(np.int16)).to(device).view(torch.bfloat16)
        elif kind == COST_SQEUCLID_F16:
            X = torch.tensor(pb.X, dtype=torch.float16, device=device)
            Y = torch.tensor(pb.Y, dtype=torch.float16, device=device)
        else:
            X = torch.tensor(pb.X, dtype=torch.float32, device=device)
            Y = torch.tensor(pb.Y, dtype=torch.float32, device=device)
        return DeviceProblem(kind, r, c, pb.s, X=X.contiguous(), Y=Y.contiguous(), cost_scale=pb.cost_scale)


@dataclasses.dataclass
class Plan:
    """Implicit rounded plan X_ij = exp(f_i + g_j - cost_scale C_ij / gamma) + kappa p_i q_j."""
    u: torch.Tensor
    v: torch.Tensor
    w: torch.Tensor
    f: torch.Tensor
    g: torch.Tensor
    p: torch.Tensor
    q: torch.Tensor
    kappa: torch.Tensor

    @staticmethod
    def empty(n: int, m: int, device="cuda") -> "Plan":
        z = lambda k: torch.zeros(k, dtype=torch.float64, device=device)
        return Plan(z(n), z(m), z(1), z(n), z(m), z(n), z(m), z(1))

    def struct(self) -> _Plan:
        s = _Plan()
        for k in ("u", "v", "w", "f", "g", "p", "q", "kappa"):
            setattr(s, k, getattr(self, k).data_ptr())
        return s


@dataclasses.dataclass
class SolveResult:
    status: int
    iters: int
    objective: float
    err_final: float
    eps_stop: float
    gamma: float
    cost_scale: float
    mass: float
    ms: float
    rounding_branch: int
    nonfinite: int
    plan: Plan
    trace: Optional[np.ndarray] = None
    pass_ms: float = 0.0
    pass_launches: int = 0
    kernel_launches: int = 0
    err_warm: float = 0.0
    err_zero: float = 0.0
    warm_used: int = 0
    tile_rows: int = 0
    tile_cols: int = 0
    tune_ms: float = 0.0
    decisions: Optional[np.ndarray] = None    # batched: per iteration took + 2 k + 8 k2 (first 1024)
    cluster_loop: int = 0                      # 1: the iterations ran in the single-cluster loop kernel


_side_streams = {}


def _stream():
    """Stream for library calls: the current torch stream, or a dedicated
    side stream when the current one is the legacy default stream (CUDA
    graphs cannot be captured on it)."""
    cur = torch.cuda.current_stream()
    if cur.cuda_stream != 0:
        return cur, None
    dev = torch.cuda.current_device()
    if dev not in _side_streams:
        _side_streams[dev] = torch.cuda.Stream()
    side = _side_streams[dev]
    side.wait_stream(cur)
    return side, cur


def _finish(side, cur):
    if cur is not None:
        cur.wait_stream(side)


def workspace_bytes(prob: DeviceProblem, flags: int = 0) -> int:
    b = ct.c_size_t(0)
    pa = _Params()
    pa.flags = flags
    _check(lib().pot_workspace_size(ct.byref(prob.struct()), ct.byref(pa), ct.byref(b)))
    return int(b.value)


def pass_kernel(prob: DeviceProblem, flags: int = 0) -> str:
    """Name of the kernel the solvers' main-loop passes run for this problem."""
    return lib().pot_pass_kernel(ct.byref(prob.struct()), int(flags)).decode()


def marginals_workspace_bytes(prob: DeviceProblem) -> int:
    """Workspace bytes of one pot_marginals pass."""
    b = ct.c_size_t(0)
    _check(lib().pot_marginals_workspace_size(ct.byref(prob.struct()), ct.byref(b)))
    return int(b.value)


_ws_cache = {}


def _workspace(prob: DeviceProblem, flags: int, ws: Optional[torch.Tensor]):
    """(buffer, usable bytes).  A caller buffer is passed with its real size
    (from its 256-byte aligned start), so the library rejects one that is
    too small instead of writing past it."""
    need = workspace_bytes(prob, flags)
    if ws is not None:
        if ws.device.type != "cuda" or not ws.is_contiguous():
            raise ValueError("workspace must be a contiguous CUDA tensor")
        nbytes = ws.numel() * ws.element_size()
        off = (-ws.data_ptr()) % 256
        if off >= nbytes:
            raise PotError(2, f"workspace too small: {nbytes} bytes < {need}")
        base = ws.view(torch.uint8)[off:]
        return base, nbytes - off
    dev = prob.r.device
    key = (dev.index, )
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < need:
        buf = torch.empty(need + 256, dtype=torch.uint8, device=dev)
        _ws_cache[key] = buf
    off = (-buf.data_ptr()) % 256
    return buf[off:], need


def _params(gamma, eps, max_iter, flags, check_every, p_tune=0.0, u0=None, v0=None, w0=0.0,
            block_rule=0, resume=None, wait_limit_ns=0) -> _Params:
    pa = _Params()
    pa.wait_limit_ns = int(wait_limit_ns)
    pa.gamma, pa.eps, pa.p_tune = float(gamma), float(eps), float(p_tune)
    pa.max_iter, pa.block_rule, pa.flags, pa.check_every = int(max_iter), int(block_rule), int(flags), int(check_every)
    pa.u0, pa.v0, pa.w0 = _ptr(u0), _ptr(v0), float(w0)
    pa._resume_ref = resume                      # keeps the state struct alive while pa is used
    pa.resume = ct.cast(ct.pointer(resume), ct.c_void_p) if resume is not None else None
    return pa


@dataclasses.dataclass
class AspotState:
    """Complete ASPOT state between iterations (z~, z_check, phi(z_check),
    theta, t): aspot_state_export fills it, aspot_solve(resume=...) goes on
    from it."""
    u_tilde: torch.Tensor
    v_tilde: torch.Tensor
    u_check: torch.Tensor
    v_check: torch.Tensor
    w_tilde: float = 0.0
    w_check: float = 0.0
    phi_check: float = 0.0
    theta: float = 1.0
    t: int = 0

    def struct(self) -> _State:
        st = _State()
        st.u_tilde, st.v_tilde = self.u_tilde.data_ptr(), self.v_tilde.data_ptr()
        st.u_check, st.v_check = self.u_check.data_ptr(), self.v_check.data_ptr()
        st.w_tilde, st.w_check, st.phi_check, st.theta = self.w_tilde, self.w_check, self.phi_check, self.theta
        st.t = int(self.t)
        return st


def aspot_state_export(prob: "DeviceProblem", ws: torch.Tensor, flags: int = 0) -> AspotState:
    """State of the last aspot_solve that ran on ``ws`` with this problem and
    these flags (pass the same ws to that solve)."""
    dev = prob.r.device
    st = AspotState(torch.empty(prob.n, dtype=torch.float64, device=dev),
                    torch.empty(prob.m, dtype=torch.float64, device=dev),
                    torch.empty(prob.n, dtype=torch.float64, device=dev),
                    torch.empty(prob.m, dtype=torch.float64, device=dev))
    raw = st.struct()
    pa = _params(1.0, 1.0, 1, flags, 0)
    base, nbytes = _workspace(prob, flags, ws)           # the same aligned start the solve used
    side, cur = _stream()
    _check(lib().aspot_state_export(ct.byref(prob.struct()), ct.byref(pa), ct.c_void_p(base.data_ptr()), nbytes,
                                    ct.byref(raw), ct.c_void_p(side.cuda_stream)))
    _finish(side, cur)
    st.w_tilde, st.w_check, st.phi_check, st.theta, st.t = raw.w_tilde, raw.w_check, raw.phi_check, raw.theta, raw.t
    return st


def _solve(fn, prob, gamma, eps, max_iter, flags, check_every, p_tune, u0, v0, w0, plan, ws,
           allow_noconv, block_rule=0, resume=None, wait_limit_ns=0) -> SolveResult:
    L = lib()
    plan = plan or Plan.empty(prob.n, prob.m, prob.r.device)
    ws, need = _workspace(prob, flags, ws)
    pa = _params(gamma, eps, max_iter, flags, check_every, p_tune, u0, v0, w0, block_rule,
                 resume.struct() if resume is not None else None, wait_limit_ns)
    res = _Result()
    side, cur = _stream()
    st = _check(getattr(L, fn)(ct.byref(prob.struct()), ct.byref(pa), ct.c_void_p(ws.data_ptr()), need,
                               ct.byref(plan.struct()), ct.byref(res), ct.c_void_p(side.cuda_stream)),
                allow=(0, 4) if allow_noconv else (0,))
    trace = None
    if flags & FLAG_TRACE:
        k = min(res.iters, 4096)
        buf = np.zeros((max(k, 1), 4))
        _check(L.pot_trace(ct.c_void_p(ws.data_ptr()), k, buf.ctypes.data_as(ct.c_void_p),
                           ct.c_void_p(side.cuda_stream)))
        trace = buf[:k]
    _finish(side, cur)
    return SolveResult(st, res.iters, res.objective, res.err_final, res.eps_stop, res.gamma, res.cost_scale,
                       res.mass, res.ms, res.rounding_branch, res.nonfinite, plan, trace,
                       res.pass_ms, res.pass_launches, res.kernel_launches, res.err_warm, res.err_zero,
                       res.warm_used, cluster_loop=res.cluster_loop)


def aspot_solve(prob: DeviceProblem, gamma: float, eps: float, max_iter: int = 10000, flags: int = 0,
                check_every: int = 0, u0=None, v0=None, w0: float = 0.0, plan: Optional[Plan] = None,
                ws: Optional[torch.Tensor] = None, allow_noconv: bool = True,
                block_rule: int = BLOCK_CYCLIC, resume: Optional["AspotState"] = None,
                wait_limit_ns: int = 0) -> SolveResult:
    """ASPOT (Algorithm 2).  block_rule: BLOCK_CYCLIC (t mod 3, Algorithm 1) or
    BLOCK_GREEDY (the block with the largest decrease of phi).  resume: go on
    from a state exported by aspot_state_export (max_iter counts from 0).
    wait_limit_ns: bound of the tcgen05 passes' pipeline waits (0: 2 s;
    negative: the stall test hook of pot_params)."""
    return _solve("aspot_solve", prob, gamma, eps, max_iter, flags, check_every, 0.0, u0, v0, w0, plan, ws,
                  allow_noconv, block_rule, resume, wait_limit_ns)


def sinkhorn_pot_solve(prob: DeviceProblem, gamma: float, eps: float, max_iter: int = 100000, flags: int = 0,
                       check_every: int = 0, p_tune: float = 0.0, plan: Optional[Plan] = None,
                       ws: Optional[torch.Tensor] = None, allow_noconv: bool = True) -> SolveResult:
    return _solve("sinkhorn_pot_solve", prob, gamma, eps, max_iter, flags, check_every, p_tune, None, None, 0.0,
                  plan, ws, allow_noconv)


def pot_round(prob: DeviceProblem, gamma: float, u: torch.Tensor, v: torch.Tensor, w: float,
              plan: Optional[Plan] = None, ws: Optional[torch.Tensor] = None):
    plan = plan or Plan.empty(prob.n, prob.m, prob.r.device)
    ws, need = _workspace(prob, 0, ws)
    br = ct.c_int32(0)
    side, cur = _stream()
    _check(lib().pot_round(ct.byref(prob.struct()), gamma, u.data_ptr(), v.data_ptr(), float(w),
                           ct.c_void_p(ws.data_ptr()), need, ct.byref(plan.struct()), ct.byref(br),
                           ct.c_void_p(side.cuda_stream)))
    _finish(side, cur)
    return plan, int(br.value)


def pot_objective(prob: DeviceProblem, plan: Plan, gamma: float, ws: Optional[torch.Tensor] = None) -> float:
    ws, need = _workspace(prob, 0, ws)
    out = ct.c_double(0)
    side, cur = _stream()
    _check(lib().pot_objective(ct.byref(prob.struct()), ct.byref(plan.struct()), gamma, ct.c_void_p(ws.data_ptr()),
                               need, ct.byref(out), ct.c_void_p(side.cuda_stream)))
    _finish(side, cur)
    return float(out.value)


def pot_marginals(prob: DeviceProblem, gamma: float, u: torch.Tensor, v: torch.Tensor, w: float,
                  ws: Optional[torch.Tensor] = None, check: bool = True, rows: bool = True, cols: bool = True):
    """Returns (log row sums, log column sums, total mass) of B(u, v, w).
    ``check``: synchronise and raise if the pass reported a stalled pipeline
    (pot_pass_status); without it the call only enqueues and the mass is
    returned as a device tensor.  ``rows`` / ``cols`` False: that side is not
    computed (returned as None); with rows=False the pass is columns-only and
    the mass is summed over the columns."""
    ws, need = _workspace(prob, 0, ws)
    lrow = torch.empty(prob.n, dtype=torch.float64, device=prob.r.device) if rows else None
    lcol = torch.empty(prob.m, dtype=torch.float64, device=prob.r.device) if cols else None
    tot = torch.empty(1, dtype=torch.float64, device=prob.r.device)
    side, cur = _stream()
    _check(lib().pot_marginals(ct.byref(prob.struct()), gamma, u.data_ptr(), v.data_ptr(), float(w),
                               ct.c_void_p(ws.data_ptr()), need, None if lrow is None else lrow.data_ptr(),
                               None if lcol is None else lcol.data_ptr(), tot.data_ptr(),
                               ct.c_void_p(side.cuda_stream)))
    if not check:
        _finish(side, cur)
        return lrow, lcol, tot
    _check(lib().pot_pass_status(ct.c_void_p(ws.data_ptr()), ct.c_void_p(side.cuda_stream)))
    _finish(side, cur)
    return lrow, lcol, float(tot.item())


def pot_cost_max(prob: DeviceProblem, ws: Optional[torch.Tensor] = None) -> float:
    ws, need = _workspace(prob, 0, ws)
    out = ct.c_double(0)
    side, cur = _stream()
    _check(lib().pot_cost_max(ct.byref(prob.struct()), ct.c_void_p(ws.data_ptr()), need, ct.byref(out),
                              ct.c_void_p(side.cuda_stream)))
    _finish(side, cur)
    return float(out.value)


def pot_plan_dense(prob: DeviceProblem, plan: Plan, gamma: float) -> torch.Tensor:
    X = torch.empty(prob.n, prob.m, dtype=torch.float32, device=prob.r.device)
    side, cur = _stream()
    _check(lib().pot_plan_dense(ct.byref(prob.struct()), ct.byref(plan.struct()), gamma, X.data_ptr(), X.stride(0),
                                ct.c_void_p(side.cuda_stream)))
    side.synchronize()
    _finish(side, cur)
    return X


def aspot_solve_batched(probs, gamma: float, eps: float, max_iter: int = 10000, flags: int = 0,
                        check_every: int = 0, plans=None, ws: Optional[torch.Tensor] = None,
                        allow_noconv: bool = True, block_rule: int = BLOCK_CYCLIC, decisions: bool = False):
    """Solve many independent squared-Euclidean problems (d <= 4) in lockstep.
    Returns one SolveResult per problem; with ``decisions`` each carries the
    per-iteration argmin and block decisions of its first 1024 iterations."""
    L = lib()
    count = len(probs)
    parr = (_Problem * count)(*[p.struct() for p in probs])
    b = ct.c_size_t(0)
    _check(L.pot_workspace_size_batched(parr, count, ct.byref(b)))
    need = int(b.value)
    dev = probs[0].r.device
    if ws is None:
        buf = torch.empty(need + 256, dtype=torch.uint8, device=dev)
        off = (-buf.data_ptr()) % 256
        ws, nbytes = buf[off:], need
    else:
        off = (-ws.data_ptr()) % 256
        ws = ws.view(torch.uint8)[off:]
        nbytes = ws.numel()
    plans = plans or [Plan.empty(p.n, p.m, dev) for p in probs]
    plarr = (_Plan * count)(*[pl.struct() for pl in plans])
    rarr = (_Result * count)()
    pa = _params(gamma, eps, max_iter, flags, check_every, block_rule=block_rule)
    side, cur = _stream()
    _check(L.aspot_solve_batched(parr, count, ct.byref(pa), ct.c_void_p(ws.data_ptr()), nbytes, plarr, rarr,
                                 ct.c_void_p(side.cuda_stream)), allow=(0, 4) if allow_noconv else (0,))
    codes = None
    if decisions:
        it = min(max(int(rarr[k].iters) for k in range(count)), 1024)
        codes = np.zeros((count, max(it, 1)), dtype=np.uint8)
        _check(L.pot_trace_batched(ct.c_void_p(ws.data_ptr()), parr, count, it, codes.ctypes.data_as(ct.c_void_p),
                                   ct.c_void_p(side.cuda_stream)))
    _finish(side, cur)
    out = []
    for k in range(count):
        r = rarr[k]
        out.append(SolveResult(r.status, r.iters, r.objective, r.err_final, r.eps_stop, r.gamma, r.cost_scale,
                               r.mass, r.ms, r.rounding_branch, r.nonfinite, plans[k], None, r.pass_ms,
                               r.pass_launches, r.kernel_launches, tile_rows=r.tile_rows, tile_cols=r.tile_cols,
                               tune_ms=r.tune_ms,
                               decisions=None if codes is None else codes[k, :min(int(r.iters), 1024)].copy()))
    return out


def _prob_array(probs):
    return (_Problem * len(probs))(*[p.struct() for p in probs])


def autotune_set(probs, tile_rows: int, tile_cols: int) -> None:
    """Pin the batched pass's tile shape for the signature of this batch."""
    _check(lib().pot_autotune_set(_prob_array(probs), len(probs), int(tile_rows), int(tile_cols)))


def autotune_lookup(probs) -> tuple:
    """Cached (tile_rows, tile_cols) for this batch's signature, (0, 0) if none."""
    h, w = ct.c_int32(0), ct.c_int32(0)
    _check(lib().pot_autotune_lookup(_prob_array(probs), len(probs), ct.byref(h), ct.byref(w)))
    return int(h.value), int(w.value)


def autotune_clear() -> None:
    _check(lib().pot_autotune_clear())


def autotune_save(path: str) -> None:
    _check(lib().pot_autotune_save(os.fsencode(path)))


def autotune_load(path: str) -> None:
    _check(lib().pot_autotune_load(os.fsencode(path)))
