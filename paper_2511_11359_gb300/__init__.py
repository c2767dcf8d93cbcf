"""Python binding of liblamp.so, the GB300 implementation of Log-Averaged Mirror Prox
(LAMP, arXiv 2511.11359) for discrete optimal transport.

The binding only marshals arguments: tensors supply device memory, the current
torch CUDA stream supplies the stream, and every step of the method runs in the
library's CUDA kernels.  There is no CPU path: importing this module on a
machine without the built library raises ImportError, and using it without a
CUDA device raises from the library.

Entry points mirror include/lamp.h:

    Lamp(...)              lamp_create            (device tensors, borrowed)
    Lamp.solve()           lamp_solve             (run Alg. 2 to the tolerance)
    Lamp.iterate(k)        lamp_iterate           (exactly k iterations)
    Lamp.objective()       lamp_objective         (<C,X>, residuals, H, P^eta, certificate, dual, K, L, gap)
    Lamp.dual()            lamp_dual              (saddle dual D at theta^t and nu^t)
    Lamp.round()           lamp_round             (Round(X^t) in factored form, its cost)
    Lamp.apply_map(V, side) lamp_apply_map        (p V or p^T U: transport-map application)
    Lamp.grad()            lamp_grad              (envelope gradient w.r.t. the points)
    Lamp.get_state()/set_state()                  (checkpoint / restore of the O(n+m) state)
    LampHost(...)          lamp_create_owned / lamp_step_host (host buffers)
    lamp_ot_loss(x, y, ...)  torch.autograd.Function with the hand-written backward
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path
from typing import Optional

import numpy as np

__all__ = [
    "LampError", "Lamp", "LampHost", "LampOT", "lamp_ot_loss", "lib", "library_path",
    "LAMP_OK", "LAMP_E_INVALID", "LAMP_E_CUDA", "LAMP_E_NOMEM", "LAMP_E_NOT_CONVERGED",
    "LAMP_E_NUMERIC", "LAMP_E_TIMEOUT", "LAMP_E_UNSUPPORTED",
    "COST_DENSE", "COST_SQEUCLID", "COST_L1", "COST_LINF", "COST_COSINE", "PREC_FP32", "PREC_BF16_TC", "EXPORTED_SYMBOLS", "selftest_wait_timeout",
]

LAMP_OK = 0
LAMP_E_INVALID = 1
LAMP_E_CUDA = 2
LAMP_E_NOMEM = 3
LAMP_E_NOT_CONVERGED = 4
LAMP_E_NUMERIC = 5
LAMP_E_TIMEOUT = 6
LAMP_E_UNSUPPORTED = 7
COST_DENSE = 0
COST_SQEUCLID = 1
COST_L1 = 2
COST_LINF = 3
COST_COSINE = 4
_POINT_COSTS = {"sqeuclid": COST_SQEUCLID, "l1": COST_L1, "linf": COST_LINF, "cosine": COST_COSINE}
PREC_FP32 = 0
PREC_BF16_TC = 1
OBJECTIVE_SLOTS = 10  # LAMP_OBJECTIVE_SLOTS of lamp.h

EXPORTED_SYMBOLS = [
    "lamp_params_default", "lamp_create", "lamp_solve", "lamp_iterate", "lamp_objective", "lamp_grad",
    "lamp_get_state", "lamp_set_state", "lamp_step_host", "lamp_create_owned",
    "lamp_launches_per_iteration", "lamp_last_error", "lamp_destroy", "lamp_time_kernels",
    "lamp_marginals_noalloc", "lamp_measure_ex2_rate", "lamp_round", "lamp_dual", "lamp_selftest_wait_timeout",
    "lamp_apply_map",
]

library_path = Path(__file__).resolve().parent / "liblamp.so"


class LampError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"LAMP error {code}: {msg}")
        self.code = code


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("d", ctypes.c_int64),
                ("kind", ctypes.c_int32), ("_pad0", ctypes.c_int32),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("r", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("cost_scale", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("tau1", ctypes.c_double), ("tau2", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int64), ("check_every", ctypes.c_int64),
                ("prec", ctypes.c_int32), ("infeas_only", ctypes.c_int32), ("K", ctypes.c_double),
                ("gap_tol", ctypes.c_double), ("gap_every", ctypes.c_int64)]


class _Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("infeas", ctypes.c_double), ("obj_CX", ctypes.c_double),
                ("kappa", ctypes.c_double), ("K", ctypes.c_double), ("status", ctypes.c_int32),
                ("stop", ctypes.c_int32), ("gap", ctypes.c_double)]


STOP_REASONS = {0: None, 1: "infeasibility", 2: "gap", 3: "max_iter"}


def _load():
    if not library_path.exists():
        raise ImportError(f"{library_path.name} is not built; run paper_2511_11359_gb300.build.build() "
                          "(nvcc for sm_103a).  There is no CPU fallback.")
    L = ctypes.CDLL(str(library_path))
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    L.lamp_params_default.argtypes = [ctypes.POINTER(_Params)]
    L.lamp_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Problem), ctypes.POINTER(_Params), vp]
    L.lamp_create_owned.argtypes = L.lamp_create.argtypes
    L.lamp_solve.argtypes = [vp, ctypes.POINTER(_Result)]
    L.lamp_iterate.argtypes = [vp, i64]
    L.lamp_objective.argtypes = [vp, ctypes.POINTER(dbl)]
    L.lamp_grad.argtypes = [vp, vp, vp]
    L.lamp_round.argtypes = [vp, ctypes.POINTER(dbl), vp, vp, vp]
    L.lamp_selftest_wait_timeout.argtypes = [i64, ctypes.POINTER(ctypes.c_int)]
    L.lamp_dual.argtypes = [vp, ctypes.POINTER(dbl)]
    L.lamp_apply_map.argtypes = [vp, vp, i64, vp, ctypes.c_int]
    L.lamp_get_state.argtypes = [vp, vp, vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(i64), vp]
    L.lamp_set_state.argtypes = [vp, vp, vp, dbl, i64, vp]
    L.lamp_step_host.argtypes = [vp, vp, vp, vp, vp, i64, ctypes.POINTER(dbl), vp]
    L.lamp_time_kernels.argtypes = [vp, i64, ctypes.POINTER(dbl)]
    L.lamp_launches_per_iteration.argtypes = [vp]
    L.lamp_launches_per_iteration.restype = i64
    L.lamp_last_error.argtypes = [vp]
    L.lamp_last_error.restype = ctypes.c_char_p
    L.lamp_destroy.argtypes = [vp]
    L.lamp_destroy.restype = None
    for name in EXPORTED_SYMBOLS:
        if name not in ("lamp_launches_per_iteration", "lamp_last_error", "lamp_destroy"):
            getattr(L, name).restype = ctypes.c_int
    return L


_LIB = None


def _get_lib():
    """Load liblamp.so on first use (so that the build step can import this package)."""
    global _LIB
    if _LIB is None:
        _LIB = _load()
    return _LIB


def __getattr__(name):
    if name == "lib":
        return _get_lib()
    raise AttributeError(name)


def _check(code: int, ctx=None, ok=(LAMP_OK,)):
    if code not in ok:
        msg = _get_lib().lamp_last_error(ctx)
        raise LampError(code, msg.decode() if msg else "")
    return code


def default_params(**kw) -> _Params:
    p = _Params()
    _check(_get_lib().lamp_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "prec" and isinstance(v, str):
            v = {"fp32": PREC_FP32, "bf16_tc": PREC_BF16_TC}[v]
        setattr(p, k, v)
    return p


def measure_ex2_rate() -> float:
    """Sustained ex2 results per SM per clock of the current device (lamp_measure_ex2_rate)."""
    v = ctypes.c_double()
    L = _get_lib()
    L.lamp_measure_ex2_rate.argtypes = [ctypes.POINTER(ctypes.c_double)]
    _check(L.lamp_measure_ex2_rate(ctypes.byref(v)))
    return v.value


def selftest_wait_timeout(polls: int) -> int:
    """Run the bounded-wait self-test (lamp_selftest_wait_timeout) and return the device
    status word it produced (LAMP_E_TIMEOUT when the wait gave up as designed)."""
    st = ctypes.c_int(0)
    _check(_get_lib().lamp_selftest_wait_timeout(int(polls), ctypes.byref(st)))
    return st.value


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class Lamp:
    """One LAMP problem on the current CUDA device (lamp_create).

    Either ``C`` (n x m float32, row-major, >= 0) or points ``x`` (n x d) and
    ``y`` (m x d) float32 CUDA tensors with a ground ``cost`` ("sqeuclid", "l1", "linf",
    "cosine"), plus float64 CUDA marginals ``r``, ``c``.
    The tensors are borrowed: this object keeps references to them.
    Keyword parameters are those of lamp_params (eta, tau1, tau2, alpha, beta,
    tol, max_iter, check_every, prec, K)."""

    def __init__(self, r, c, *, x=None, y=None, C=None, cost_scale: float = 1.0, cost: str = "sqeuclid",
                 stream=None, **params):
        import torch

        self._keep = [r, c, x, y, C]
        for t in (r, c):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("r and c must be contiguous float64 CUDA tensors")
        prob = _Problem()
        prob.n = r.shape[0]
        prob.m = c.shape[0]
        if C is not None:
            if C.dtype != torch.float32 or not C.is_cuda or C.stride(1) != 1:
                raise ValueError("C must be a float32 CUDA tensor with unit column stride")
            prob.kind = COST_DENSE
            prob.C = _ptr(C)
            prob.ldc = C.stride(0)
            prob.d = 0
            if tuple(C.shape) != (prob.n, prob.m):
                raise ValueError("C must be n x m")
        else:
            for t in (x, y):
                if t is None or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                    raise ValueError("x and y must be contiguous float32 CUDA tensors")
            if cost not in _POINT_COSTS:
                raise ValueError(f"cost must be one of {sorted(_POINT_COSTS)}")
            prob.kind = _POINT_COSTS[cost]
            prob.x = _ptr(x)
            prob.y = _ptr(y)
            prob.d = x.shape[1]
            if x.shape[0] != prob.n or y.shape[0] != prob.m or y.shape[1] != prob.d:
                raise ValueError("x must be n x d and y m x d")
        prob.r = _ptr(r)
        prob.c = _ptr(c)
        prob.cost_scale = float(cost_scale)
        self.n, self.m, self.d = int(prob.n), int(prob.m), int(prob.d)
        self.kind = prob.kind
        self.params = default_params(**params)
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        _check(_get_lib().lamp_create(ctypes.byref(h), ctypes.byref(prob), ctypes.byref(self.params),
                               ctypes.c_void_p(stream.cuda_stream)))
        self._h = h

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            _get_lib().lamp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- Alg. 2
    def solve(self, allow_not_converged: bool = True) -> dict:
        res = _Result()
        ok = (LAMP_OK, LAMP_E_NOT_CONVERGED) if allow_not_converged else (LAMP_OK,)
        code = _check(_get_lib().lamp_solve(self._h, ctypes.byref(res)), self._h, ok)
        return {"iters": int(res.iters), "infeas": res.infeas, "cost": res.obj_CX, "kappa": res.kappa,
                "K": res.K, "status": int(res.status), "converged": code == LAMP_OK,
                "stop": STOP_REASONS.get(int(res.stop)), "gap": res.gap}

    def iterate(self, k: int) -> None:
        _check(_get_lib().lamp_iterate(self._h, int(k)), self._h)

    def objective(self) -> dict:
        out = (ctypes.c_double * OBJECTIVE_SLOTS)()
        _check(_get_lib().lamp_objective(self._h, out), self._h)
        keys = ["cost", "col_res", "row_res", "entropy", "P_eta", "certificate", "dual", "K", "L", "gap"]
        return dict(zip(keys, list(out)))

    def dual(self) -> dict:
        """D(theta^t), D(nu^t): the saddle-problem dual at both potentials (App. B)."""
        out = (ctypes.c_double * 2)()
        _check(_get_lib().lamp_dual(self._h, out), self._h)
        return {"theta": out[0], "nu": out[1]}

    def apply_map(self, V, side: int = 0):
        """p V (side 0, V: m x k) or p^T U (side 1, U: n x k) for the current X^t = diag(r) p
        (lamp_apply_map); V a device float32 tensor with 1 <= k <= 8 columns."""
        import torch

        V = V.contiguous()
        if V.dim() == 1:
            V = V[:, None]
        rows = self.n if side == 0 else self.m
        out = torch.empty((rows, V.shape[1]), dtype=torch.float32, device=V.device)
        _check(_get_lib().lamp_apply_map(self._h, ctypes.c_void_p(_ptr(V)), int(V.shape[1]),
                                         ctypes.c_void_p(_ptr(out)), int(side)), self._h)
        return out

    def round(self, want_vectors: bool = False) -> dict:
        """Round(X^t) = X^t diag(y) + dr dc^T / ||dr||_1 (Alg. 3): its cost and, with
        want_vectors, the device float64 tensors y (m), dr (n), dc (m)."""
        import torch

        dev = torch.device("cuda", torch.cuda.current_device())
        vec = {}
        if want_vectors:
            vec = {"y": torch.empty(self.m, dtype=torch.float64, device=dev),
                   "dr": torch.empty(self.n, dtype=torch.float64, device=dev),
                   "dc": torch.empty(self.m, dtype=torch.float64, device=dev)}
        out = (ctypes.c_double * 4)()
        _check(_get_lib().lamp_round(self._h, out, ctypes.c_void_p(_ptr(vec.get("y"))),
                                     ctypes.c_void_p(_ptr(vec.get("dr"))), ctypes.c_void_p(_ptr(vec.get("dc")))),
               self._h)
        res = {"cost": out[0], "dr_l1": out[1], "dc_l1": out[2], "cost_scaled": out[3]}
        res.update(vec)
        return res

    def grad(self, want_x: bool = True, want_y: bool = True):
        import torch

        dev = torch.device("cuda", torch.cuda.current_device())
        dx = torch.empty((self.n, self.d), dtype=torch.float32, device=dev) if want_x else None
        dy = torch.empty((self.m, self.d), dtype=torch.float32, device=dev) if want_y else None
        _check(_get_lib().lamp_grad(self._h, ctypes.c_void_p(_ptr(dx)), ctypes.c_void_p(_ptr(dy))), self._h)
        return dx, dy

    def get_state(self) -> dict:
        nu = np.empty(self.m)
        th = np.empty(self.m)
        lz = np.empty(self.n)
        rs = np.empty(2 * self.n, dtype=np.float32)
        kap = ctypes.c_double()
        t = ctypes.c_int64()
        _check(_get_lib().lamp_get_state(self._h, nu.ctypes.data, th.ctypes.data, lz.ctypes.data,
                                  ctypes.byref(kap), ctypes.byref(t), rs.ctypes.data), self._h)
        return {"nu": nu, "theta": th, "logZ": lz, "kappa": kap.value, "t": t.value, "row_shifts": rs}

    def set_state(self, nu, theta, kappa: float, t: int, row_shifts=None) -> None:
        nu = np.ascontiguousarray(nu, dtype=np.float64)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        rs = None if row_shifts is None else np.ascontiguousarray(row_shifts, dtype=np.float32)
        _check(_get_lib().lamp_set_state(self._h, nu.ctypes.data, th.ctypes.data, float(kappa), int(t),
                                  None if rs is None else rs.ctypes.data), self._h)

    def time_kernels(self, iters: int) -> list:
        """Run `iters` iterations kernel by kernel with CUDA events between the
        launches; mean ms of [row sweep, row finalize, column sweep, column finalize]."""
        out = (ctypes.c_double * 4)()
        _check(_get_lib().lamp_time_kernels(self._h, int(iters), out), self._h)
        return list(out)

    def launches_per_iteration(self) -> int:
        return int(_get_lib().lamp_launches_per_iteration(self._h))


class LampHost:
    """A context that owns device copies of host (NumPy) inputs: lamp_create_owned,
    then lamp_step_host, which re-uploads the inputs, iterates and reads back."""

    def __init__(self, r, c, *, x=None, y=None, C=None, cost_scale: float = 1.0, stream=None, **params):
        import torch

        self.r = np.ascontiguousarray(r, dtype=np.float64)
        self.c = np.ascontiguousarray(c, dtype=np.float64)
        prob = _Problem()
        prob.n, prob.m = self.r.shape[0], self.c.shape[0]
        if C is not None:
            self.a = np.ascontiguousarray(C, dtype=np.float32)
            self.b = None
            prob.kind, prob.C, prob.ldc, prob.d = COST_DENSE, self.a.ctypes.data, prob.m, 0
        else:
            self.a = np.ascontiguousarray(x, dtype=np.float32)
            self.b = np.ascontiguousarray(y, dtype=np.float32)
            prob.kind, prob.x, prob.y, prob.d = COST_SQEUCLID, self.a.ctypes.data, self.b.ctypes.data, self.a.shape[1]
        prob.r, prob.c, prob.cost_scale = self.r.ctypes.data, self.c.ctypes.data, float(cost_scale)
        self.n, self.m = int(prob.n), int(prob.m)
        self.params = default_params(**params)
        if stream is None:
            stream = torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(_get_lib().lamp_create_owned(ctypes.byref(h), ctypes.byref(prob), ctypes.byref(self.params),
                                     ctypes.c_void_p(stream.cuda_stream)))
        self._h = h

    def step(self, iters: int, a=None, b=None, r=None, c=None, nu_out: Optional[np.ndarray] = None) -> float:
        a = self.a if a is None else a
        b = self.b if b is None else b
        r = self.r if r is None else r
        c = self.c if c is None else c
        inf = ctypes.c_double()
        _check(_get_lib().lamp_step_host(self._h, a.ctypes.data, 0 if b is None else b.ctypes.data, r.ctypes.data,
                                  c.ctypes.data, int(iters), ctypes.byref(inf),
                                  0 if nu_out is None else nu_out.ctypes.data), self._h)
        return inf.value

    def close(self):
        if getattr(self, "_h", None):
            _get_lib().lamp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_loss_function():
    import torch

    class LampOT(torch.autograd.Function):
        """Forward: solve the OT problem between point clouds with LAMP (lamp_create /
        lamp_solve / lamp_objective) and return L = <C,X> - eta H(X).
        Backward: lamp_grad (envelope gradient dL/dx_i = sum_j X_ij dC_ij/dx_i, one
        fused recompute pass, X never stored) times the incoming gradient."""

        @staticmethod
        def forward(ctx, x, y, r, c, eta, cost_scale, params):
            solver = Lamp(r, c, x=x.detach().contiguous(), y=y.detach().contiguous(), cost_scale=cost_scale,
                          eta=eta, **params)
            info = solver.solve()
            obj = solver.objective()
            ctx.solver = solver
            ctx.info = info
            ctx.obj = obj
            return torch.tensor(obj["L"], dtype=torch.float64, device=x.device)

        @staticmethod
        def backward(ctx, g):
            dx, dy = ctx.solver.grad(ctx.needs_input_grad[0], ctx.needs_input_grad[1])
            ctx.solver.close()
            gs = g.to(torch.float32)
            return (None if dx is None else dx * gs, None if dy is None else dy * gs, None, None, None, None, None)

    return LampOT


try:
    LampOT = _make_loss_function()
except ImportError:  # torch unavailable: only the ctypes layer is usable
    LampOT = None


def lamp_ot_loss(x, y, r=None, c=None, eta: float = 1e-2, cost_scale: float = 1.0, **params):
    """Differentiable entropic OT loss between float32 CUDA point clouds x (n x d), y (m x d)."""
    import torch

    if r is None:
        r = torch.full((x.shape[0],), 1.0 / x.shape[0], dtype=torch.float64, device=x.device)
    if c is None:
        c = torch.full((y.shape[0],), 1.0 / y.shape[0], dtype=torch.float64, device=y.device)
    return LampOT.apply(x, y, r, c, float(eta), float(cost_scale), params)
