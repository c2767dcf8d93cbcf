"""FP64 CPU oracle of Log-Averaged Mirror Prox (LAMP), arXiv 2511.11359.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import
this module.  The product path (the CUDA library and its Python binding) never
imports it and shares no code with it.

Everything here is plain, dense, float64 NumPy written from the paper's
definitions and algorithms, in the paper's order and notation:

  K      = ||C||_inf = max_ij |C_ij|                                (Section 2)
  kappa  = 1/eta_t, kappa_0 = 0 (eta_0 = infinity)                  (Alg. 2)
  p^eta(nu)_ij = exp(-(C_ij + 2K nu_j)/eta) / Z_i                   (Eq. def:dual_to_primal)
  log Z_i = LSE_j(-kappa (C_ij + 2K nu_j))                          (Section 4.1)
  col_r(p) = col(diag(r) p)                                         (Section 2.2)
  dual mirror map  tanh(2 tau K / c^alpha (col - c) + atanh theta0) (Eq. def:closed_form_opt)
  tclip(theta, beta) = clip to [-tanh(beta/2), tanh(beta/2)]       (Section 3.1)

Readings of passages that are silent, ambiguous or garbled:
  * kappa_0 = 0 stands for eta_0 = infinity, so X^0 = diag(r) (1/m).
  * beta defaults to 1.1 (App. E.2), the clip bound is tanh(0.55).
  * tau1 = tau2 = 1/(2K) and alpha = 0.01 by default, for eta = 0 and eta > 0.
  * infeasibility = ||col(X^t) - c||_1 + ||row(X^t) - r||_1 on X^t (not the
    midpoint), summed in float64.
  * the eta > 0 saddle dual D^eta includes the constant -eta H(r) that the
    printed formula (App. B) omits, so that weak duality holds as stated.

Functions whose result has no independent pin would be marked "parity unpinned"; none
is (``Dt_summand`` is pinned by the re-expression in tests/test_oracle_dt.py).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

__all__ = [
    "LampParams", "LampState", "StepInfo",
    "sqeuclid_cost", "l1_cost", "linf_cost", "cosine_cost", "cost_matrix", "sup_norm",
    "kappa_next", "kappa_closed_form", "log_normalizers", "dual_to_primal", "col_r", "row_sums",
    "dual_mirror_map", "tclip", "calpha_of", "resolve_params",
    "lamp_initial_state", "lamp_step", "lamp_run", "lamp_solve",
    "lamp_performant_run", "pdmp_run", "primal_mirror_map",
    "round_plan", "round_factors", "entropy", "penalized_objective", "entropy_from_normalizers",
    "saddle_dual", "certificate_rhs", "objective_report",
    "sinkhorn_log", "eot_value", "ot_lp", "ot_bruteforce_uniform",
    "grad_envelope", "D_Ha", "KL", "Dt_summand",
    "logZ_rows", "col_entries", "marginals_from_state",
    "sqeuclid_cost_expanded", "lamp_step_streamed", "streamed_sup_norm",
]


# --------------------------------------------------------------------------------------
# cost


def sqeuclid_cost(x: np.ndarray, y: np.ndarray, scale: float = 1.0, chunk: int = 256) -> np.ndarray:
    """C_ij = scale * sum_k (x_ik - y_jk)^2 in float64 from the given coordinates
    (the l2^2 ground cost of Section 5), by explicit differences, row chunk by row chunk."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.shape[0]
    out = np.empty((n, y.shape[0]), dtype=np.float64)
    for a in range(0, n, chunk):
        diff = x[a:a + chunk, None, :] - y[None, :, :]
        out[a:a + chunk] = (diff * diff).sum(axis=2)
    if scale != 1.0:
        out *= scale
    return out


def l1_cost(x: np.ndarray, y: np.ndarray, scale: float = 1.0) -> np.ndarray:
    """C_ij = scale * sum_k |x_ik - y_jk| (the l1 ground cost of App. E.2), in float64."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros((x.shape[0], y.shape[0]))
    for k in range(x.shape[1]):
        out += np.abs(x[:, None, k] - y[None, :, k])
    return out * scale


def linf_cost(x: np.ndarray, y: np.ndarray, scale: float = 1.0) -> np.ndarray:
    """C_ij = scale * max_k |x_ik - y_jk| (the l-infinity ground cost of App. E.2), in float64."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros((x.shape[0], y.shape[0]))
    for k in range(x.shape[1]):
        out = np.maximum(out, np.abs(x[:, None, k] - y[None, :, k]))
    return out * scale


def cosine_cost(x: np.ndarray, y: np.ndarray, scale: float = 1.0) -> np.ndarray:
    """C_ij = scale * (1 - <x_i, y_j> / (|x_i| |y_j|)) (the cosine ground cost of App. E.2), in float64."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    nx = np.sqrt((x * x).sum(axis=1))
    ny = np.sqrt((y * y).sum(axis=1))
    return (1.0 - (x @ y.T) / (nx[:, None] * ny[None, :])) * scale


def sqeuclid_cost_expanded(x: np.ndarray, y: np.ndarray, scale: float = 1.0) -> np.ndarray:
    """The same C_ij = scale |x_i - y_j|^2 in float64 written as |x_i|^2 + |y_j|^2 - 2 x_i . y_j
    (a matrix product), for row blocks of large high-dimensional clouds where the
    explicit differences would need n m d memory.  Agrees with sqeuclid_cost to
    float64 rounding (pinned by a test)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    C = (x * x).sum(axis=1)[:, None] + (y * y).sum(axis=1)[None, :] - 2.0 * (x @ y.T)
    np.maximum(C, 0.0, out=C)
    if scale != 1.0:
        C *= scale
    return C


def sup_norm(C: np.ndarray) -> float:
    """||C||_inf = max_ij |C_ij| (Section 2, entry-wise matrix norm)."""
    return float(np.max(np.abs(C)))


def cost_matrix(workload) -> np.ndarray:
    """The float64 cost the oracle solves for a workload: the stored float32
    matrix as is, or the squared Euclidean cost of the float32 points.  A
    negative cost_scale divides by the maximum cost (normalised cost)."""
    if workload.kind == "dense":
        return np.asarray(workload.C, dtype=np.float64)
    C = sqeuclid_cost(workload.x, workload.y)
    s = workload.cost_scale
    if s < 0:
        C /= C.max()
    elif s != 1.0:
        C *= s
    return C


# --------------------------------------------------------------------------------------
# the building blocks of Alg. 2


def kappa_next(kappa: float, eta: float, tau1: float) -> float:
    """1/eta_{t+1} = tau1 + (1/eta_t)(1 - tau1 eta): the reciprocal form of the
    eta_t recursion of Alg. 2 (Section 3.2), with kappa = 1/eta_t."""
    return tau1 + kappa * (1.0 - tau1 * eta)


def kappa_closed_form(t: int, eta: float, tau1: float) -> float:
    """Solved recursion (Section 3.2): 1/eta_t = (1 - (1 - tau1 eta)^t)/eta, and
    1/eta_t = tau1 t in the limit eta -> 0."""
    if eta == 0.0:
        return tau1 * t
    return (1.0 - (1.0 - tau1 * eta) ** t) / eta


def log_normalizers(C: np.ndarray, K: float, kappa: float, nu: np.ndarray) -> np.ndarray:
    """log Z_i = LSE_j(-kappa (C_ij + 2K nu_j)) by the max-shifted LSE of Section 4.1."""
    S = -kappa * (C + 2.0 * K * nu[None, :])
    mx = S.max(axis=1)
    return mx + np.log(np.exp(S - mx[:, None]).sum(axis=1))


def dual_to_primal(C: np.ndarray, K: float, kappa: float, nu: np.ndarray):
    """p^eta(nu) = diag(Z)^{-1} exp(-kappa (C + 2K 1 nu^T)) (Eq. def:dual_to_primal,
    kappa = 1/eta; kappa = 0 gives the uniform rows of the eta_0 = infinity start).
    Returns (p, log Z)."""
    logZ = log_normalizers(C, K, kappa, nu)
    S = -kappa * (C + 2.0 * K * nu[None, :])
    return np.exp(S - logZ[:, None]), logZ


def col_r(p: np.ndarray, r: np.ndarray) -> np.ndarray:
    """col_r(p) = col(diag(r) p) (Section 2.2)."""
    return (r[:, None] * p).sum(axis=0)


def row_sums(X: np.ndarray) -> np.ndarray:
    return X.sum(axis=1)


def calpha_of(c: np.ndarray, alpha: float) -> np.ndarray:
    """c^alpha = c + (alpha/m) 1 (Section 3.1)."""
    return c + alpha / c.shape[0]


def dual_mirror_map(theta0: np.ndarray, colr: np.ndarray, c: np.ndarray, calpha: np.ndarray,
                    tau: float, K: float) -> np.ndarray:
    """Dual mirror map in closed form (Eq. def:closed_form_opt, second line):
    tanh(2 tau K / c^alpha_j (col_r(p)_j - c_j) + (1/2) log((1+theta0_j)/(1-theta0_j)))."""
    return np.tanh(2.0 * tau * K / calpha * (colr - c) + 0.5 * np.log((1.0 + theta0) / (1.0 - theta0)))


def tclip(theta: np.ndarray, beta: float) -> np.ndarray:
    """Coordinate-wise clip to [-tanh(beta/2), tanh(beta/2)] (Section 3.1)."""
    b = np.tanh(beta / 2.0)
    return np.clip(theta, -b, b)


@dataclass
class LampParams:
    """Alg. 2 inputs.  tau1/tau2 = None means 1/(2K); K = None means ||C||_inf
    (App. E.2 defaults: alpha = 0.01, beta = 1.1)."""
    eta: float = 0.0
    tau1: Optional[float] = None
    tau2: Optional[float] = None
    alpha: float = 0.01
    beta: float = 1.1
    K: Optional[float] = None


def resolve_params(C: np.ndarray, params: LampParams):
    K = sup_norm(C) if params.K is None else float(params.K)
    tau1 = 1.0 / (2.0 * K) if params.tau1 is None else float(params.tau1)
    tau2 = 1.0 / (2.0 * K) if params.tau2 is None else float(params.tau2)
    if tau1 * params.eta > 1.0:
        raise ValueError("Alg. 2 needs tau1 * eta <= 1")
    return K, tau1, tau2


@dataclass
class LampState:
    """The whole O(m) state of Alg. 2 at the start of iteration t."""
    t: int
    kappa: float
    nu: np.ndarray
    theta: np.ndarray

    def copy(self) -> "LampState":
        return LampState(self.t, self.kappa, self.nu.copy(), self.theta.copy())


@dataclass
class StepInfo:
    """What one iteration of Alg. 2 computes besides the new state.

    A = col(X^t), X^t = diag(r) p^{eta_t}(nu^t); B = col(Xbar^{t+1}),
    Xbar^{t+1} = diag(r) p^{eta_{t+1}}(nubar^{t+1}); logZ_A, logZ_B their row
    normalisers; cost_A = <C, X^t>; res = ||A - c||_1 + ||row(X^t) - r||_1."""
    A: np.ndarray
    B: np.ndarray
    logZ_A: np.ndarray
    logZ_B: np.ndarray
    cost_A: float
    res: float
    row_res: float
    nubar: np.ndarray
    thetabar: np.ndarray
    thetahat: np.ndarray
    kappa_next: float


def lamp_initial_state(m: int) -> LampState:
    """theta^0 = nu^0 = 0, eta_0 = infinity (Alg. 2)."""
    return LampState(0, 0.0, np.zeros(m), np.zeros(m))


def lamp_step(C, r, c, K, tau1, tau2, eta, calpha, beta, state: LampState):
    """One iteration t of Alg. 2 (Step 1), in the order the algorithm states it."""
    kap = state.kappa
    nu = state.nu
    theta = state.theta
    # eta_{t+1} = eta_t / (1 + tau1 (eta_t - eta)), kept as its reciprocal
    kap1 = kappa_next(kap, eta, tau1)
    w = tau1 / kap1                                   # tau1 * eta_{t+1}
    # nubar^{t+1} = nu^t + tau1 eta_{t+1} (theta^t - nu^t)
    nubar = nu + w * (theta - nu)
    # thetabar^{t+1} = M_{tau2}(theta^t; p^{eta_t}(nu^t))
    pA, logZ_A = dual_to_primal(C, K, kap, nu)
    XA = r[:, None] * pA
    A = XA.sum(axis=0)
    thetabar = dual_mirror_map(theta, A, c, calpha, tau2, K)
    # nu^{t+1} = nu^t + tau1 eta_{t+1} (thetabar^{t+1} - nu^t)
    nu_new = nu + w * (thetabar - nu)
    # thetahat^{t+1} = M_{tau2}(theta^t; p^{eta_{t+1}}(nubar^{t+1}))
    pB, logZ_B = dual_to_primal(C, K, kap1, nubar)
    B = col_r(pB, r)
    thetahat = dual_mirror_map(theta, B, c, calpha, tau2, K)
    # theta^{t+1} = tclip(thetahat^{t+1}, beta)
    theta_new = tclip(thetahat, beta)
    row_res = float(np.abs(XA.sum(axis=1) - r).sum())
    info = StepInfo(A=A, B=B, logZ_A=logZ_A, logZ_B=logZ_B, cost_A=float((C * XA).sum()),
                    res=float(np.abs(A - c).sum()) + row_res, row_res=row_res,
                    nubar=nubar, thetabar=thetabar, thetahat=thetahat, kappa_next=kap1)
    new_state = LampState(state.t + 1, kap1, nu_new, theta_new)
    return new_state, info


def lamp_run(C, r, c, params: LampParams, T: int, state: Optional[LampState] = None,
             record: Optional[Callable[[LampState, StepInfo], None]] = None) -> LampState:
    """Run exactly T iterations of Alg. 2 from ``state`` (default: the Alg. 2 start)."""
    C = np.asarray(C, dtype=np.float64)
    K, tau1, tau2 = resolve_params(C, params)
    calpha = calpha_of(c, params.alpha)
    st = lamp_initial_state(C.shape[1]) if state is None else state.copy()
    for _ in range(T):
        prev = st
        st, info = lamp_step(C, r, c, K, tau1, tau2, params.eta, calpha, params.beta, st)
        if record is not None:
            record(prev, info)
    return st


def lamp_solve(C, r, c, params: LampParams, tol: float, max_iter: int,
               state: Optional[LampState] = None):
    """Iterate Alg. 2 until X^t meets the termination rule, checked on X^t before
    the iteration's updates: the first t >= 1 with infeasibility <= tol (App. E.2)
    and, for eta > 0, 1 - kappa_t eta <= tol (kappa_t -> 1/eta, Section 3.2, so that
    X^t solves the eta problem and not the one of eta_t).  t = 0 is excluded: the
    start X^0 = diag(r)/m is exactly feasible whenever c is uniform, and the
    certificate of Prop. infeas_bound (a) is stated for t >= 1.

    Returns (state_t, info_t, converged): the state whose X^t met the rule (or the
    state after max_iter iterations) and its StepInfo."""
    C = np.asarray(C, dtype=np.float64)
    K, tau1, tau2 = resolve_params(C, params)
    calpha = calpha_of(c, params.alpha)
    st = lamp_initial_state(C.shape[1]) if state is None else state.copy()
    info = None
    for _ in range(max_iter + 1):
        nxt, info = lamp_step(C, r, c, K, tau1, tau2, params.eta, calpha, params.beta, st)
        kappa_ok = params.eta == 0.0 or 1.0 - st.kappa * params.eta <= tol
        if st.t >= 1 and info.res <= tol and kappa_ok:
            return st, info, True
        if st.t >= max_iter:
            break
        st = nxt
    return st, info, False


# --------------------------------------------------------------------------------------
# Alg. 4 (performant parameters) and Alg. 1 (explicit PDMP), used as cross-checks


def lamp_performant_run(C, r, c, alpha: float, T: int, record=None):
    """Alg. 4 (App. D): eta = 0, tau1 = tau2 = 1/(2K), clip to [-1/2, 1/2], with
    p^{eta_t}(nu)_ij proportional to exp(-t (C_ij/(2K) + nu_j)) and the dual
    argmax steps solved through grad H_c^alpha(theta) = c^alpha atanh(theta)."""
    C = np.asarray(C, dtype=np.float64)
    K = sup_norm(C)
    n, m = C.shape
    ca = c + alpha / m
    nu = np.zeros(m)
    theta = np.zeros(m)
    Ch = C / (2.0 * K)
    for t in range(T):
        nubar = t / (t + 1.0) * nu + theta / (t + 1.0)
        E = -t * (Ch + nu[None, :])
        E -= E.max(axis=1, keepdims=True)
        P = np.exp(E)
        P /= P.sum(axis=1, keepdims=True)
        A = (r[:, None] * P).sum(axis=0)
        # argmax <A - c, th> - D_Ha(th || theta): c^alpha (atanh th - atanh theta) = A - c
        thetabar = np.tanh(np.arctanh(theta) + (A - c) / ca)
        nu_new = t / (t + 1.0) * nu + thetabar / (t + 1.0)
        E = -(t + 1.0) * (Ch + nubar[None, :])
        E -= E.max(axis=1, keepdims=True)
        P = np.exp(E)
        P /= P.sum(axis=1, keepdims=True)
        B = (r[:, None] * P).sum(axis=0)
        thetahat = np.tanh(np.arctanh(theta) + (B - c) / ca)
        theta = np.clip(thetahat, -0.5, 0.5)
        nu = nu_new
        if record is not None:
            record(t, nu, theta, A, B)
    return nu, theta


def primal_mirror_map(logp0: np.ndarray, C: np.ndarray, K: float, theta: np.ndarray,
                      tau: float, eta: float) -> np.ndarray:
    """Primal mirror map in closed form (Eq. def:closed_form_opt, first line), in
    logs: log p+ = (1 - tau eta) log p0 - tau (C + 2K theta) - log Z."""
    L = (1.0 - tau * eta) * logp0 - tau * (C + 2.0 * K * theta[None, :])
    mx = L.max(axis=1, keepdims=True)
    return L - (mx + np.log(np.exp(L - mx).sum(axis=1, keepdims=True)))


def pdmp_run(C, r, c, params: LampParams, T: int, record=None):
    """Alg. 1 (explicit PDMP) with O(nm) primal iterates kept as log p.
    record(t, p^t, pbar^{t+1}, theta^t) is called each iteration."""
    C = np.asarray(C, dtype=np.float64)
    K, tau1, tau2 = resolve_params(C, params)
    n, m = C.shape
    ca = calpha_of(c, params.alpha)
    logp = np.full((n, m), -np.log(m))
    theta = np.zeros(m)
    for t in range(T):
        p = np.exp(logp)
        logpbar = primal_mirror_map(logp, C, K, theta, tau1, params.eta)
        thetabar = dual_mirror_map(theta, col_r(p, r), c, ca, tau2, K)
        logp_new = primal_mirror_map(logp, C, K, thetabar, tau1, params.eta)
        thetahat = dual_mirror_map(theta, col_r(np.exp(logpbar), r), c, ca, tau2, K)
        if record is not None:
            record(t, p, np.exp(logpbar), theta)
        theta = tclip(thetahat, params.beta)
        logp = logp_new
    return np.exp(logp), theta


# --------------------------------------------------------------------------------------
# Round, objectives, duals, certificate


def round_factors(X: np.ndarray, r: np.ndarray, c: np.ndarray):
    """Alg. 3 (Round, Altschuler et al.), steps 1-3: the row scaling x, the column
    scaling y, X'' = diag(x) X diag(y), and delta_r = r - row(X''),
    delta_c = c - col(X'').  Returns (x, y, X'', delta_r, delta_c)."""
    x = np.minimum(r / X.sum(axis=1), 1.0)
    X1 = x[:, None] * X
    y = np.minimum(c / X1.sum(axis=0), 1.0)
    X2 = X1 * y[None, :]
    dr = r - X2.sum(axis=1)
    dc = c - X2.sum(axis=0)
    return x, y, X2, dr, dc


def round_plan(X: np.ndarray, r: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Alg. 3 (Round), step 4 on the factors of round_factors: X'' plus the rank-one
    correction delta_r delta_c^T / ||delta_r||_1.  With ||delta_r||_1 = 0 the
    correction is skipped (X'' is already feasible up to rounding)."""
    _, _, X2, dr, dc = round_factors(X, r, c)
    l1 = np.abs(dr).sum()
    if l1 == 0.0:
        return X2
    return X2 + np.outer(dr, dc) / l1


def entropy(X: np.ndarray) -> float:
    """H(X) = -<X, log X> with 0 log 0 = 0 (Section 2)."""
    Xp = X[X > 0]
    return float(-(Xp * np.log(Xp)).sum())


def penalized_objective(X, C, c, K, eta) -> float:
    """P^eta(X) = <C,X> + 2||C||_inf ||col(X) - c||_1 - eta H(X) (Eq. prob:l1_ot_primal)."""
    return float((C * X).sum() + 2.0 * K * np.abs(X.sum(axis=0) - c).sum() - eta * entropy(X))


def entropy_from_normalizers(r, logZ, kappa, K, cost, colX, nu) -> float:
    """H(X) from O(n+m) quantities for X = diag(r) p^{1/kappa}(nu):
    H(X) = H(r) + kappa <C,X> + 2 K kappa <col(X), nu> + <r, log Z>.
    This is the identity of the lemma in App. D (there with K = 1,
    kappa = t/2), written for any kappa."""
    Hr = -float((r * np.log(r)).sum())
    return Hr + kappa * cost + 2.0 * K * kappa * float(colX @ nu) + float(r @ logZ)


def saddle_dual(C, r, c, K, theta, eta: float = 0.0) -> float:
    """Dual of the saddle problem (App. B): eta = 0 gives
    D(theta) = sum_i r_i min_j (C_ij + 2K theta_j) - 2K <c, theta>;
    eta > 0 replaces the row min by the row softmin -eta log sum_j exp(-z_ij/eta)
    and includes the constant -eta H(r) (see the module header)."""
    Z = C + 2.0 * K * theta[None, :]
    if eta == 0.0:
        rowpart = Z.min(axis=1)
        const = 0.0
    else:
        mn = Z.min(axis=1)
        rowpart = mn - eta * np.log(np.exp(-(Z - mn[:, None]) / eta).sum(axis=1))
        const = -eta * (-(r * np.log(r)).sum())
    return float(r @ rowpart - 2.0 * K * (c @ theta) + const)


def certificate_rhs(K: float, col_res: float, m: int, t: int) -> float:
    """Right-hand side of Prop. infeas_bound (a): 4K ||col(X^t) - c||_1 + 2K log m / t."""
    return 4.0 * K * col_res + 2.0 * K * np.log(m) / t


def objective_report(C, r, c, K, eta, state: LampState) -> dict:
    """The quantities lamp_objective reports, computed densely from X^t."""
    p, logZ = dual_to_primal(C, K, state.kappa, state.nu)
    X = r[:, None] * p
    colX = X.sum(axis=0)
    cost = float((C * X).sum())
    col_res = float(np.abs(colX - c).sum())
    row_res = float(np.abs(X.sum(axis=1) - r).sum())
    H = entropy(X)
    out = {
        "cost": cost, "col_res": col_res, "row_res": row_res, "entropy": H,
        "P_eta": penalized_objective(X, C, c, K, eta),
        "L": eot_value(C, X, eta),
        "certificate": certificate_rhs(K, col_res, C.shape[1], state.t) if (eta == 0.0 and state.t > 0) else float("nan"),
        "dual": max(saddle_dual(C, r, c, K, state.theta, eta), saddle_dual(C, r, c, K, state.nu, eta)),
        "K": K, "logZ": logZ, "col": colX, "X": X,
    }
    return out


# --------------------------------------------------------------------------------------
# reference solvers that pin the oracle: Sinkhorn, LP, brute force


def sinkhorn_log(C, r, c, eta: float, tol: float = 1e-13, max_iter: int = 200000,
                 f0=None, g0=None):
    """Log-domain Sinkhorn for min_{X in Pi(r,c)} <C,X> - eta H(X) (Eq. prob:primal_eot);
    X_ij = exp((f_i + g_j - C_ij)/eta).  Alternating exact row / column fits until
    the column marginal error (rows are exact after each f update) is below tol.
    Returns (X, f, g, iterations)."""
    C = np.asarray(C, dtype=np.float64)
    n, m = C.shape
    lr = np.log(r)
    lc = np.log(c)
    f = np.zeros(n) if f0 is None else f0.copy()
    g = np.zeros(m) if g0 is None else g0.copy()
    for it in range(1, max_iter + 1):
        Mf = (g[None, :] - C) / eta
        mx = Mf.max(axis=1)
        f = eta * (lr - (mx + np.log(np.exp(Mf - mx[:, None]).sum(axis=1))))
        Mg = (f[:, None] - C) / eta
        mx = Mg.max(axis=0)
        g = eta * (lc - (mx + np.log(np.exp(Mg - mx[None, :]).sum(axis=0))))
        if it % 10 == 0 or it == max_iter:
            X = np.exp((f[:, None] + g[None, :] - C) / eta)
            err = np.abs(X.sum(axis=1) - r).sum()
            if err <= tol:
                return X, f, g, it
    X = np.exp((f[:, None] + g[None, :] - C) / eta)
    return X, f, g, max_iter


def eot_value(C, X, eta) -> float:
    return float((C * X).sum() - eta * entropy(X))


def ot_lp(C, r, c) -> float:
    """Exact OT value min_{X in Pi(r,c)} <C,X> (Eq. prob:primal_ot) by linear programming (HiGHS)."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix, vstack

    C = np.asarray(C, dtype=np.float64)
    n, m = C.shape
    idx = np.arange(n * m)
    Arow = coo_matrix((np.ones(n * m), (idx // m, idx)), shape=(n, n * m))
    Acol = coo_matrix((np.ones(n * m), (idx % m, idx)), shape=(m, n * m))
    A = vstack([Arow, Acol]).tocsr()
    b = np.concatenate([r, c])
    res = linprog(C.ravel(), A_eq=A, b_eq=b, bounds=(0, None), method="highs",
                  options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    if not res.success:
        raise RuntimeError(res.message)
    return float(res.fun)


def ot_bruteforce_uniform(C) -> float:
    """Exact OT for uniform marginals on n = m points: by Birkhoff's theorem an
    optimal plan is a permutation matrix / n, so OT = min_sigma sum_i C_{i sigma(i)} / n."""
    C = np.asarray(C, dtype=np.float64)
    n = C.shape[0]
    best = np.inf
    rows = np.arange(n)
    for perm in itertools.permutations(range(n)):
        v = C[rows, perm].sum()
        if v < best:
            best = v
    return float(best / n)


def grad_envelope(x, y, X, scale: float = 1.0):
    """Envelope gradient of L = <C,X> - eta H(X) at the optimal plan for
    C_ij = scale |x_i - y_j|^2: dL/dx_i = sum_j X_ij 2 scale (x_i - y_j),
    dL/dy_j = sum_i X_ij 2 scale (y_j - x_i)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    rowX = X.sum(axis=1)
    colX = X.sum(axis=0)
    dx = 2.0 * scale * (rowX[:, None] * x - X @ y)
    dy = 2.0 * scale * (colX[:, None] * y - X.T @ x)
    return dx, dy


# --------------------------------------------------------------------------------------
# divergences and the D_t diagnostic of Prop. infeas_bound (b)


def D_Ha(theta, nu, calpha) -> float:
    """Bregman divergence of the dual entropy H_c^alpha (Eq. def:DHa_explicit)."""
    a = (1.0 + theta) / 2.0 * np.log((1.0 + theta) / (1.0 + nu))
    b = (1.0 - theta) / 2.0 * np.log((1.0 - theta) / (1.0 - nu))
    return float(calpha @ (a + b))


def KL(X, Y) -> float:
    """KL(X||Y) = D_{-H}(X||Y) = sum X log(X/Y) - sum X + sum Y."""
    mask = X > 0
    return float((X[mask] * np.log(X[mask] / Y[mask])).sum() - X.sum() + Y.sum())


def Dt_summand(C, r, K, calpha, prev: LampState, info: StepInfo, new: LampState) -> float:
    """One summand of D_t (Eq. def:sum_condition): the D_Ha and KL differences of the
    midpoint analysis (Lemma summability).  Pinned by an independent re-expression of
    both differences (Bregman form of D_Ha; log-normaliser form of the KL difference)."""
    Xs = r[:, None] * dual_to_primal(C, K, prev.kappa, prev.nu)[0]
    Xbar = r[:, None] * dual_to_primal(C, K, info.kappa_next, info.nubar)[0]
    Xnew = r[:, None] * dual_to_primal(C, K, new.kappa, new.nu)[0]
    return (D_Ha(info.thetabar, info.thetahat, calpha) - D_Ha(info.thetabar, prev.theta, calpha)
            + KL(Xbar, Xnew) - KL(Xbar, Xs))


# --------------------------------------------------------------------------------------
# sampled evaluation at sizes where a dense n x m matrix is too large


def logZ_rows(cost_rows: Callable[[np.ndarray], np.ndarray], rows: np.ndarray, K: float,
              kappa: float, nu: np.ndarray) -> np.ndarray:
    """log Z_i for selected rows, with cost_rows(rows) returning C[rows, :] in float64."""
    Cr = cost_rows(rows)
    return log_normalizers(Cr, K, kappa, nu)


def col_entries(cost_rows: Callable[[np.ndarray], np.ndarray], n: int, cols: np.ndarray,
                K: float, kappa: float, nu: np.ndarray, r: np.ndarray, chunk: int = 512):
    """col_j of X = diag(r) p^{1/kappa}(nu) for selected columns j, streaming row
    chunks of C so that memory stays O(chunk * m).  Returns (col[cols], logZ)."""
    out = np.zeros(len(cols))
    logZ = np.empty(n)
    for a in range(0, n, chunk):
        rows = np.arange(a, min(n, a + chunk))
        Cr = cost_rows(rows)
        lz = log_normalizers(Cr, K, kappa, nu)
        logZ[rows] = lz
        S = -kappa * (Cr[:, cols] + 2.0 * K * nu[None, cols])
        out += (r[rows, None] * np.exp(S - lz[:, None])).sum(axis=0)
    return out, logZ


def streamed_sup_norm(cost_rows: Callable[[np.ndarray], np.ndarray], n: int, chunk: int = 512) -> float:
    """||C||_inf over row blocks of a cost too large to hold (Section 2)."""
    K = 0.0
    for a in range(0, n, chunk):
        K = max(K, float(np.abs(cost_rows(np.arange(a, min(n, a + chunk)))).max()))
    return K


def lamp_step_streamed(cost_rows: Callable[[np.ndarray], np.ndarray], n: int, r, c, K, tau1, tau2, eta, calpha,
                       beta, state: LampState, chunk: int = 512):
    """One iteration of Alg. 2 with C streamed in row blocks (O(chunk * m) memory):
    the same steps as lamp_step, with the two marginals (Section 4.1) accumulated
    block by block.  Returns (new_state, (A, B, logZ_A, logZ_B))."""
    m = c.shape[0]
    kap = state.kappa
    nu = state.nu
    theta = state.theta
    kap1 = kappa_next(kap, eta, tau1)
    w = tau1 / kap1
    nubar = nu + w * (theta - nu)
    cols = np.arange(m)
    A, logZ_A = col_entries(cost_rows, n, cols, K, kap, nu, r, chunk)
    thetabar = dual_mirror_map(theta, A, c, calpha, tau2, K)
    nu_new = nu + w * (thetabar - nu)
    B, logZ_B = col_entries(cost_rows, n, cols, K, kap1, nubar, r, chunk)
    thetahat = dual_mirror_map(theta, B, c, calpha, tau2, K)
    theta_new = tclip(thetahat, beta)
    return LampState(state.t + 1, kap1, nu_new, theta_new), (A, B, logZ_A, logZ_B)


def marginals_from_state(C, r, K, kappa, nu):
    """(col(X), log Z) of X = diag(r) p^{1/kappa}(nu) for a dense C."""
    p, logZ = dual_to_primal(C, K, kappa, nu)
    return col_r(p, r), logZ
