"""Helpers shared by the GPU parity tests: build solvers on identical seeded inputs
and run the FP64 oracle beside them.

Tolerances (the targets stated for this path, written out once here):
  POT_TOL   potentials nu, theta (in (-1, 1)): max |gpu - oracle| <= 1e-5
  LOGZ_TOL  log Z: |gpu - oracle| <= 1e-5 (1 + |log Z|)
  OBJ_TOL   <C, X>: relative 1e-6
  GRAD_TOL  gradients: relative (max-norm) 1e-4
  RES_FLOOR absolute noise of an L1 residual built from float32 column sums: each
            entry 2^{v} carries ~2^-22 (ex2.approx) + |v| 2^-24 ln 2 relative error,
            so sum_j |col_j - c_j| is known to ~1e-7; comparisons add 2e-7.
  On-the-fly costs: the kernels see C~ = C + delta with |delta| ~ float32 rounding of
  the cost; at kappa the exponents then differ by kappa |delta|, so comparisons at
  large kappa use cost_slack(), derived from the float32 cost of the same points.
"""
import numpy as np

import oracle as O
import workloads as W

POT_TOL = 1e-5
LOGZ_TOL = 1e-5
OBJ_TOL = 1e-6
GRAD_TOL = 1e-4
RES_FLOOR = 2e-7


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_cost(w):
    """(C64, cost_scale for the GPU, K): the oracle's float64 cost of the workload,
    the positive scale that makes the GPU solve the same cost, and ||C||_inf."""
    if w.kind == "dense":
        C = np.asarray(w.C, dtype=np.float64)
        return C, 1.0, float(C.max())
    cost = {"sqeuclid": O.sqeuclid_cost, "l1": O.l1_cost, "linf": O.linf_cost, "cosine": O.cosine_cost}[w.kind]
    D = cost(w.x, w.y)
    s = w.cost_scale
    if s < 0:
        s = 1.0 / D.max()
    elif s == 0:
        s = 1.0
    C = D * s
    return C, s, float(C.max())


def gpu_solver(w, K=None, scale=None, **params):
    import paper_2511_11359_gb300 as L

    C, s, Kref = oracle_cost(w)
    K = Kref if K is None else K
    r, c = dev(w.r), dev(w.c)
    if w.kind == "dense":
        return L.Lamp(r, c, C=dev(w.C), K=K, **params), C, K
    return L.Lamp(r, c, x=dev(w.x), y=dev(w.y), cost_scale=s if scale is None else scale, K=K, cost=w.kind,
                  **params), C, K


def gpu_solver_raw(w, K, scale=1.0, **params):
    """The GPU context for workload w with an explicit K and cost scale, without
    materialising the oracle's dense cost (for the full-size point clouds)."""
    import paper_2511_11359_gb300 as L

    r, c = dev(w.r), dev(w.c)
    if w.kind == "dense":
        return L.Lamp(r, c, C=dev(w.C), K=K, **params)
    return L.Lamp(r, c, x=dev(w.x), y=dev(w.y), cost_scale=scale, K=K, cost=w.kind, **params)


def assert_pot_close(st, ref, tol=POT_TOL, what=""):
    dn = np.abs(st["nu"] - ref.nu).max()
    dt = np.abs(st["theta"] - ref.theta).max()
    assert dn <= tol and dt <= tol, f"{what}: |dnu|={dn:.3e} |dtheta|={dt:.3e} (tol {tol:.0e})"


def assert_logZ_close(lz, ref, tol=LOGZ_TOL, what=""):
    err = np.abs(lz - ref) / (1.0 + np.abs(ref))
    assert np.all(np.isfinite(lz)), what
    assert err.max() <= tol, f"{what}: log Z rel err {err.max():.3e}"


def cost_error(w):
    """max_ij |C32_ij - C_ij|: float32 evaluation of the point cost against float64
    (|x - y|^2 by its differences; l1 / l-inf / cosine by a bound of d float32 roundings
    of terms of the cost's size)."""
    if w.kind == "dense":
        return 0.0
    if w.kind != "sqeuclid":
        C, s, K = oracle_cost(w)
        return float(2.0 * max(w.d, 2) * 2.0 ** -24 * K)
    x32 = np.asarray(w.x, np.float32)
    y32 = np.asarray(w.y, np.float32)
    d32 = np.zeros((x32.shape[0], y32.shape[0]), np.float32)
    for k in range(x32.shape[1]):
        df = x32[:, None, k] - y32[None, :, k]
        d32 += df * df
    C64 = O.sqeuclid_cost(w.x, w.y)
    _, s, _ = oracle_cost(w)
    return float(np.abs(d32.astype(np.float64) - C64).max() * s)


def cost_slack(w, kappa):
    """Potential tolerance widened by the float32 cost error at kappa (see module doc)."""
    return POT_TOL + 4.0 * kappa * cost_error(w)
