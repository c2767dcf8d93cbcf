"""Ground costs other than |x - y|^2 (App. E.2: l1, l-infinity, cosine) through the C ABI
against the FP64 oracle on the same points: trajectories of Alg. 2, the objective, Round,
the dual bound and the transport map."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_util import (OBJ_TOL, POT_TOL, RES_FLOOR, assert_logZ_close, assert_pot_close, cost_slack,
                            gpu_solver, gpu_solver_raw, oracle_cost)

pytestmark = pytest.mark.gpu

CASES = [
    # (cost, n, m, d, dist, eta, prec): packed direct sweeps (d <= 8), scalar direct form
    # (d > 8, l1 / l-inf), dot form and tensor cores (cosine)
    ("l1", 300, 257, 2, "uniform", 0.0, "fp32"),
    ("l1", 700, 1100, 3, "uniform", 0.02, "fp32"),
    ("linf", 257, 300, 3, "uniform", 0.0, "fp32"),
    ("linf", 160, 140, 12, "gauss_shift", 0.0, "fp32"),
    ("l1", 150, 170, 20, "gauss_shift", 0.05, "fp32"),
    ("cosine", 300, 280, 5, "gauss_shift", 0.0, "fp32"),
    ("cosine", 200, 230, 40, "gauss_shift", 0.0, "fp32"),
    ("cosine", 256, 200, 64, "gauss_shift", 0.0, "bf16_tc"),
]


def _problem(case):
    cost, n, m, d, dist, eta, prec = case
    w = W.points_problem(f"{cost}{d}", n, m, d, seed=n + 7 * d, dist=dist, marg="random", cost_scale=1.0, eta=eta)
    if prec == "bf16_tc":
        # points of norm exactly 1/sqrt(2) with bf16-exact coordinates: the unit scaling and
        # the bf16 rounding are exact, so the tensor cores solve the oracle's problem
        return dataclasses.replace(w, kind="cosine", x=W.half_norm_points(n, d, seed=n + 1),
                                   y=W.half_norm_points(m, d, seed=m + 2))
    return dataclasses.replace(w, kind=cost)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-d{c[3]}-{c[6]}" for c in CASES])
def test_cost_trajectory_and_evaluations(case):
    import torch

    cost, n, m, d, dist, eta, prec = case
    w = _problem(case)
    C, s, K = oracle_cost(w)
    sol, _, _ = gpu_solver(w, K=K, scale=s, eta=eta, prec=prec, check_every=7)
    P = O.LampParams(eta=eta, K=K)
    done, ref = 0, None
    for T in (1, 10, 60):
        sol.iterate(T - done)
        ref = O.lamp_run(C, w.r, w.c, P, T - done, state=ref)
        done = T
        assert_pot_close(sol.get_state(), ref, tol=cost_slack(w, ref.kappa), what=f"{case} T={T}")
    rep = O.objective_report(C, w.r, w.c, K, eta, ref)
    obj = sol.objective()
    slack = 4 * ref.kappa * 2.0 * max(d, 2) * 2.0 ** -24 * K  # exponent error of the float32 cost
    assert abs(obj["cost"] - rep["cost"]) <= (OBJ_TOL + slack) * abs(rep["cost"])
    assert abs(obj["col_res"] - rep["col_res"]) <= (1e-5 + slack) * rep["col_res"] + RES_FLOOR
    assert_logZ_close(sol.get_state()["logZ"], rep["logZ"], tol=1e-5 + slack, what=f"{case} logZ")
    # Round (Alg. 3): cost of the rounded plan
    X = rep["X"]
    Xr = O.round_plan(X, w.r, w.c)
    rd = sol.round()
    ref_cost = float((C * Xr).sum())
    assert abs(rd["cost"] - ref_cost) <= (OBJ_TOL + slack) * ref_cost + 4 * K * RES_FLOOR
    # dual bound at theta^T and nu^T (App. B)
    D = sol.dual()
    for key, phi in (("theta", ref.theta), ("nu", ref.nu)):
        refD = O.saddle_dual(C, w.r, w.c, K, phi, eta)
        assert abs(D[key] - refD) <= 2e-6 * K + 4 * K * (POT_TOL + slack), (key, D[key], refD)
    # transport map p V
    p = X / w.r[:, None]
    V = np.random.default_rng(5).uniform(-1, 1, size=(m, 2)).astype(np.float32)
    out = sol.apply_map(torch.from_numpy(V).cuda(), side=0).cpu().numpy()
    refV = p @ V.astype(np.float64)
    assert np.abs(out - refV).max() <= (1e-5 + slack) * np.abs(refV).max() + 2 * POT_TOL
    sol.close()


def test_cost_kinds_rejected_where_unsupported():
    import paper_2511_11359_gb300 as L

    w = dataclasses.replace(W.points_problem("l1rej", 40, 30, 3, seed=2), kind="l1")
    s, _, _ = gpu_solver(w)
    with pytest.raises(L.LampError):
        s.grad()
    s.close()
    with pytest.raises(L.LampError):
        gpu_solver(w, prec="bf16_tc")
    z = W.points_problem("cosrej", 40, 30, 3, seed=3)
    z.x[5] = 0.0  # a zero point has no cosine
    with pytest.raises(L.LampError):
        gpu_solver_raw(dataclasses.replace(z, kind="cosine"), K=1.0)
