"""lamp_round (Alg. 3), lamp_dual (App. B, Eqs. def:dual_spp / def:dual_spp_e) and
lamp_apply_map (App. E colour transfer) through the C ABI against the FP64 oracle.

The GPU context is put on the oracle's own state at iteration T (lamp_set_state with
the oracle's nu, theta, kappa), so both sides evaluate the same X^T; the oracle rounds
the dense X^T (round_factors / round_plan) and evaluates saddle_dual densely."""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_util import OBJ_TOL, RES_FLOOR, gpu_solver, oracle_cost

pytestmark = pytest.mark.gpu

CASES = [
    # (name, kind, n, m, d, eta, prec, T): direct-form and dot-form float32 sweeps, the
    # tcgen05 path on bf16-rounded points, stored costs; ragged sizes spanning several
    # CTAs and inner splits
    ("pts2", "points", 300, 257, 2, 0.0, "fp32", 40),
    ("pts3_eta", "points", 1500, 1100, 3, 0.05, "fp32", 25),
    ("dense", "dense", 290, 1100, 0, 0.0, "fp32", 30),
    ("dense_eta", "dense", 700, 300, 0, 0.02, "fp32", 20),
    # stored cost whose TMA-fed column sweep splits its rows over 4 CTAs per column block
    ("dense_split", "dense", 1024, 512, 0, 0.0, "fp32", 20),
    ("dot16", "points", 400, 300, 16, 0.0, "fp32", 30),
    ("tc64", "points", 384, 300, 64, 0.0, "bf16_tc", 30),
]


def _problem(case):
    name, kind, n, m, d, eta, prec, T = case
    seed = sum(name.encode()) % 991
    if kind == "dense":
        return W.dense_problem(name, n, m, seed=seed, eta=eta)
    dist = "gauss_shift" if d > 8 else "uniform"
    w = W.points_problem(name, n, m, d, seed=seed, dist=dist, marg="random", cost_scale=1.0, eta=eta)
    if prec == "bf16_tc":
        w = dataclasses.replace(w, x=W.bf16_round(w.x), y=W.bf16_round(w.y))
    return w


def _setup(case):
    name, kind, n, m, d, eta, prec, T = case
    w = _problem(case)
    C, s, K = oracle_cost(w)
    st = O.lamp_run(C, w.r, w.c, O.LampParams(eta=eta, K=K), T)
    sol, _, _ = gpu_solver(w, K=K, scale=s, eta=eta, prec=prec, check_every=5)
    sol.set_state(st.nu, st.theta, st.kappa, st.t)
    return w, C, s, K, st, sol


def _dot_slack(w, s):
    """float32 error of an on-the-fly cost in the dot form (d > 8, or bf16 inputs):
    d accumulated roundings of terms of size up to s (|x|^2 + |y|^2)."""
    if w.kind == "dense" or w.d <= 8:
        return 0.0
    nx = (np.asarray(w.x, np.float64) ** 2).sum(1).max()
    ny = (np.asarray(w.y, np.float64) ** 2).sum(1).max()
    return w.d * 2.0 ** -24 * s * (nx + ny)


def _cost_err(w, s):
    """Bound on max_ij |C~_ij - C_ij| of the kernels' float32 cost: 0 for a stored cost,
    the float32 evaluation of the squared differences (direct form, d <= 8), the dot-form
    bound otherwise."""
    if w.kind == "dense":
        return 0.0
    if w.d > 8:
        return _dot_slack(w, s)
    from tests.gpu_util import cost_error

    return cost_error(w)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_round_matches_oracle(case):
    w, C, s, K, st, sol = _setup(case)
    g = sol.round(want_vectors=True)
    X = w.r[:, None] * O.dual_to_primal(C, K, st.kappa, st.nu)[0]
    x, y, X2, dr, dc = O.round_factors(X, w.r, w.c)
    assert np.abs(x - 1.0).max() <= 1e-12  # row(X^t) = r: Step 1 is the identity
    Xr = O.round_plan(X, w.r, w.c)
    ref_cost = float((C * Xr).sum())
    ref_cpp = float((C * X2).sum())
    slack = _dot_slack(w, s)
    gy, gdr, gdc = (g[k].cpu().numpy() for k in ("y", "dr", "dc"))
    assert np.abs(gy - y).max() <= 1e-5, np.abs(gy - y).max()
    assert np.all(np.abs(gdc - dc) <= 1e-5 * w.c + 1e-9)
    assert np.abs(gdr - dr).sum() <= 1e-5 * np.abs(dr).sum() + RES_FLOOR
    assert np.all(gdr >= 0.0) and np.all(gdc >= 0.0)
    assert abs(g["dr_l1"] - np.abs(dr).sum()) <= 1e-5 * np.abs(dr).sum() + RES_FLOOR
    assert abs(g["dc_l1"] - np.abs(dc).sum()) <= 1e-5 * np.abs(dc).sum() + RES_FLOOR
    # mass balance: sum delta_r = sum delta_c = 1 - mass(X'')
    assert abs(g["dr_l1"] - g["dc_l1"]) <= 2 * RES_FLOOR
    assert abs(g["cost_scaled"] - ref_cpp) <= OBJ_TOL * abs(ref_cpp) + slack
    assert abs(g["cost"] - ref_cost) <= OBJ_TOL * abs(ref_cost) + 4 * K * RES_FLOOR + slack
    # the factored plan is feasible: col = y * col(X^t) + delta_c = c (checked on the oracle's col)
    colX = X.sum(axis=0)
    assert np.abs(gy * colX + gdc - w.c).max() <= 2e-5 * w.c.max()
    sol.close()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_dual_matches_oracle(case):
    name, kind, n, m, d, eta, prec, T = case
    w, C, s, K, st, sol = _setup(case)
    D = sol.dual()
    ref_t = O.saddle_dual(C, w.r, w.c, K, st.theta, eta)
    ref_n = O.saddle_dual(C, w.r, w.c, K, st.nu, eta)
    # D is 1-Lipschitz in the cost (max norm): the kernels' float32 cost differs from the
    # oracle's by at most the cost error bound; beyond it, eta = 0 is exact to ~1e-12 K
    # (two row-max passes) and eta > 0 carries the ex2 error, ~2^-22 eta
    tol = 1e-9 * K + 2.0 * _cost_err(w, s) + (4e-7 * eta if eta > 0 else 0.0)
    assert abs(D["theta"] - ref_t) <= tol, (D["theta"], ref_t, tol)
    assert abs(D["nu"] - ref_n) <= tol, (D["nu"], ref_n, tol)
    obj = sol.objective()
    assert obj["dual"] == max(D["theta"], D["nu"])
    assert obj["gap"] == pytest.approx(obj["P_eta"] - obj["dual"], rel=0, abs=1e-12 * K)
    sol.close()


EXACT_CASES = [
    # points on a 1/16 grid: every squared distance (direct form) and every x.y (dot form,
    # bf16 tensor cores included) is exact in float32, so the kernels' cost is the oracle's
    ("dy3", 300, 257, 3, "fp32"),
    ("dy16", 400, 300, 16, "fp32"),
    ("dy64tc", 384, 300, 64, "bf16_tc"),
    ("dense_exact", 290, 1100, 0, "fp32"),
]


@pytest.mark.parametrize("case", EXACT_CASES, ids=[c[0] for c in EXACT_CASES])
def test_dual_is_exact_on_an_exact_cost(case):
    """eta = 0 dual D(phi) (Eq. def:dual_spp) on costs the float32 kernels represent exactly:
    |D_gpu - D_oracle| <= 1e-9 K at theta^T and nu^T."""
    name, n, m, d, prec = case
    seed = sum(name.encode()) % 991
    if d == 0:
        w = W.dense_problem(name, n, m, seed=seed)
    else:
        dist = "gauss_shift" if d > 8 else "uniform"
        w = W.points_problem(name, n, m, d, seed=seed, dist=dist, marg="random", cost_scale=1.0, grid_step=16)
    C, s, K = oracle_cost(w)
    st = O.lamp_run(C, w.r, w.c, O.LampParams(K=K), 60)
    sol, _, _ = gpu_solver(w, K=K, scale=s, prec=prec, check_every=5)
    sol.set_state(st.nu, st.theta, st.kappa, st.t)
    D = sol.dual()
    for key, phi in (("theta", st.theta), ("nu", st.nu)):
        ref = O.saddle_dual(C, w.r, w.c, K, phi, 0.0)
        assert abs(D[key] - ref) <= 1e-9 * K, (name, key, D[key] - ref)
    sol.close()


def test_round_dual_and_certificate_bracket_the_lp_optimum():
    """eta = 0 on an LP-sized problem after T iterations: weak duality D(theta^T) <= OT*
    (App. B), Round(X^T) is feasible so <C, Round(X^T)> >= OT*, and Prop. infeas_bound (a)
    bounds <C, Round(X^T)> - OT* by the certificate 4K ||col - c||_1 + 2K log m / T."""
    w = W.points_problem("lpbracket", 40, 36, 2, seed=5, dist="uniform", marg="random", cost_scale=1.0)
    C, s, K = oracle_cost(w)
    ot = O.ot_lp(C, w.r, w.c)
    sol, _, _ = gpu_solver(w, K=K, scale=s, check_every=10)
    for T in (20, 200):
        sol.iterate(T - (0 if T == 20 else 20))
        obj = sol.objective()
        rd = sol.round()
        D = sol.dual()
        assert max(D["theta"], D["nu"]) <= ot + 1e-9 * K + 2.0 * _cost_err(w, s)
        assert rd["cost"] >= ot - OBJ_TOL * ot
        assert rd["cost"] - ot <= obj["certificate"] + OBJ_TOL * ot
        assert obj["certificate"] == pytest.approx(4 * K * obj["col_res"] + 2 * K * math.log(w.m) / T, rel=1e-12)
    sol.close()


def test_round_leaves_the_state_alone():
    """lamp_round and lamp_dual use only scratch buffers: the trajectory after them is the
    trajectory without them, bit for bit."""
    w = W.points_problem("roundstate", 257, 300, 3, seed=11, dist="uniform", marg="random", cost_scale=1.0)
    C, s, K = oracle_cost(w)
    a, _, _ = gpu_solver(w, K=K, scale=s, check_every=4)
    b, _, _ = gpu_solver(w, K=K, scale=s, check_every=4)
    a.iterate(13)
    b.iterate(13)
    b.round(want_vectors=True)
    b.dual()
    a.iterate(9)
    b.iterate(9)
    sa, sb = a.get_state(), b.get_state()
    assert np.array_equal(sa["nu"], sb["nu"]) and np.array_equal(sa["theta"], sb["theta"])
    assert np.array_equal(sa["row_shifts"], sb["row_shifts"])
    a.close()
    b.close()


MAP_CASES = [
    # (case of CASES, k)
    (CASES[0], 3), (CASES[1], 1), (CASES[2], 8), (CASES[3], 2), (CASES[4], 5), (CASES[5], 3),
]


@pytest.mark.parametrize("case,kv", MAP_CASES, ids=[f"{c[0]}-k{k}" for c, k in MAP_CASES])
def test_apply_map_matches_oracle(case, kv):
    """lamp_apply_map: p V and p^T U (App. E colour transfer) against the dense oracle p."""
    import torch

    w, C, s, K, st, sol = _setup(case)
    p = O.dual_to_primal(C, K, st.kappa, st.nu)[0]
    rng = np.random.default_rng(kv + w.n)
    V = rng.uniform(-1.0, 1.0, size=(w.m, kv)).astype(np.float32)
    U = rng.uniform(0.0, 1.0, size=(w.n, kv)).astype(np.float32)
    out0 = sol.apply_map(torch.from_numpy(V).cuda(), side=0).cpu().numpy().astype(np.float64)
    out1 = sol.apply_map(torch.from_numpy(U).cuda(), side=1).cpu().numpy().astype(np.float64)
    ref0 = p @ V.astype(np.float64)
    ref1 = p.T @ U.astype(np.float64)
    # exponent error of the on-the-fly float32 cost at kappa_T (dot form), see _dot_slack
    rel = 1e-5 + 4.0 * st.kappa * _dot_slack(w, s)
    assert np.abs(out0 - ref0).max() <= rel * np.abs(ref0).max(), np.abs(out0 - ref0).max()
    assert np.abs(out1 - ref1).max() <= rel * np.abs(ref1).max(), np.abs(out1 - ref1).max()
    # p is row-stochastic, and p^T r = col(diag(r) p)
    ones = sol.apply_map(torch.ones((w.m, 1), dtype=torch.float32, device="cuda"), side=0).cpu().numpy()
    assert np.abs(ones - 1.0).max() <= 1e-6
    colr = sol.apply_map(torch.from_numpy(w.r.astype(np.float32)[:, None]).cuda(), side=1).cpu().numpy()[:, 0]
    colX = (w.r[:, None] * p).sum(axis=0)
    assert np.abs(colr - colX).max() <= rel * colX.max()
    sol.close()


@pytest.mark.parametrize("eta", [0.0, 0.05])
def test_solve_stops_on_the_primal_dual_gap(eta):
    """gap_tol > 0: lamp_solve stops at the first evaluated X^t whose primal-dual gap
    P^eta(X^t) - max D (App. B duals, App. E.2 termination) is <= gap_tol, with the
    infeasibility rule off (tol = 0).  The gap then certifies the optimum: by weak duality
    and Lemma l1_prob_equiv, D <= OT* (EOT*) <= P^eta, checked against the LP (eta = 0) and
    FP64 Sinkhorn (eta > 0) on a cost the kernels represent exactly (points on a 1/16 grid).
    The float32 primal is known to ~1e-7 K, so the tolerance is 1e-6 K, not the 1e-10 of the
    paper's FP64 runs."""
    w = W.points_problem("gap", 40, 36, 2, seed=5, dist="uniform", marg="random", cost_scale=1.0, eta=eta,
                         grid_step=16)
    C, s, K = oracle_cost(w)
    if eta == 0.0:
        ref = O.ot_lp(C, w.r, w.c)
    else:
        ref = O.eot_value(C, O.sinkhorn_log(C, w.r, w.c, eta, tol=1e-14)[0], eta)
    gap_tol = 1e-6 * K
    sol, _, _ = gpu_solver(w, K=K, scale=s, eta=eta, tol=0.0, max_iter=400000, check_every=100,
                           gap_tol=gap_tol, gap_every=500)
    res = sol.solve(allow_not_converged=False)
    assert res["stop"] == "gap" and res["gap"] <= gap_tol, res
    obj = sol.objective()  # the same state: the same gap
    assert obj["gap"] == pytest.approx(res["gap"], rel=0, abs=1e-12 * K)
    # the dual's own error: ~1e-12 K at eta = 0, the ex2 error ~2^-22 eta of the softmin at eta > 0
    assert obj["dual"] <= ref + 1e-9 * K + 4e-7 * eta, (obj["dual"], ref)
    assert ref <= obj["P_eta"] + 2e-7 * K, (obj["P_eta"], ref)
    assert obj["P_eta"] - ref <= gap_tol + 1e-9 * K
    sol.close()
    # gap_tol = 0 keeps the infeasibility rule alone
    sol2, _, _ = gpu_solver(w, K=K, scale=s, eta=eta, tol=1e-5, max_iter=400000, check_every=10,
                            infeas_only=1)
    r2 = sol2.solve(allow_not_converged=False)
    assert r2["stop"] == "infeasibility" and r2["infeas"] <= 1e-5 and np.isnan(r2["gap"])
    sol2.close()
