"""The GPU path at the full sizes of the five workloads, against the FP64 oracle.

Each test runs the oracle's own trajectory from the Alg. 2 start (no GPU value is
ever an oracle input); where a dense n x m cost is too large for the host, the
oracle streams C in row blocks (lamp_step_streamed) or checks sampled rows and
properties that hold at any size."""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_util import (GRAD_TOL, LOGZ_TOL, OBJ_TOL, POT_TOL, RES_FLOOR, assert_logZ_close, assert_pot_close,
                            dev, gpu_solver, gpu_solver_raw, oracle_cost)

pytestmark = pytest.mark.gpu


def _expanded_rows(x, y):
    x64 = np.asarray(x, np.float64)
    y64 = np.asarray(y, np.float64)
    return lambda rows: O.sqeuclid_cost_expanded(x64[rows], y64)


@pytest.mark.parametrize("prec,T", [("bf16_tc", 2), ("fp32", 1)])
def test_highdim_fullsize_iterations(prec, T):
    """n = m = 2^15, d = 64 (the bench workload, same launch configuration): T
    iterations of Alg. 2 and the evaluation of X^T, all m potentials and all n
    log-normalisers against the streamed oracle (bf16: on the rounded points)."""
    w = W.highdim()
    if prec == "bf16_tc":
        w = dataclasses.replace(w, x=W.bf16_round(w.x), y=W.bf16_round(w.y))
    rows = _expanded_rows(w.x, w.y)
    K = O.streamed_sup_norm(rows, w.n, chunk=1024)
    P = O.LampParams(K=K)
    K_, tau1, tau2 = O.resolve_params(np.zeros((1, 1)), P)
    ca = O.calpha_of(w.c, P.alpha)
    st = O.lamp_initial_state(w.m)
    for _ in range(T):
        st, _ = O.lamp_step_streamed(rows, w.n, w.r, w.c, K, tau1, tau2, 0.0, ca, P.beta, st, chunk=1024)
    colT, logZT = O.col_entries(rows, w.n, np.arange(w.m), K, st.kappa, st.nu, w.r, chunk=1024)

    s = gpu_solver_raw(w, K, 1.0, prec=prec, check_every=50)
    s.iterate(T)
    obj = s.objective()
    g = s.get_state()
    assert g["t"] == T
    assert_pot_close(g, st, what=f"highdim {prec} T={T}")
    assert_logZ_close(g["logZ"], logZT, what=f"highdim {prec} log Z")
    assert abs(obj["col_res"] - np.abs(colT - w.c).sum()) <= 1e-6 * np.abs(colT - w.c).sum() + RES_FLOOR
    s.close()


def test_largescale_fullsize_first_iterate():
    """n = m = 2^18, d = 3: after one iteration nu^1 has a closed form (col(X^0) = 1/m,
    w = 1: nu^1 = tanh(2 tau2 K / c^alpha (1/m - c))), so nu^1 is checked on all m
    entries and log Z of X^1 on sampled rows; the context's device memory is O(n + m)."""
    import torch

    w = W.largescale()
    Kp = 3.0  # an upper bound of |x - y|^2 on [0,1]^3, given to both sides
    free0 = torch.cuda.mem_get_info()[0]
    s = gpu_solver_raw(w, Kp, 1.0, check_every=1)
    ctx_bytes = free0 - torch.cuda.mem_get_info()[0]
    s.iterate(1)
    obj = s.objective()
    g = s.get_state()
    P = O.LampParams(K=Kp)
    K_, tau1, tau2 = O.resolve_params(np.zeros((1, 1)), P)
    ca = O.calpha_of(w.c, P.alpha)
    nu1 = 0.0 + (tau1 / O.kappa_next(0.0, 0.0, tau1)) * (
        O.dual_mirror_map(np.zeros(w.m), np.full(w.m, 1.0 / w.m), w.c, ca, tau2, Kp) - 0.0)
    assert np.abs(g["nu"] - nu1).max() <= POT_TOL
    assert np.all(np.abs(g["theta"]) <= math.tanh(0.55) + 1e-15)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(w.n, 64, replace=False))
    x64 = w.x.astype(np.float64)
    lz = O.logZ_rows(lambda rr: O.sqeuclid_cost(x64[rr], w.y, chunk=8), rows, Kp, g["kappa"], nu1)
    assert g["kappa"] == pytest.approx(tau1, rel=1e-15)
    assert_logZ_close(g["logZ"][rows], lz, what="largescale log Z rows")
    assert 0.0 <= obj["cost"] <= Kp and np.isfinite(obj["col_res"])
    # O(n + m) device memory: a few hundred bytes per support point
    assert ctx_bytes <= 512 * (w.n + w.m), ctx_bytes
    s.close()


def test_image_grid_fullsize_trajectory():
    """n = m = 4096 stored cost (64 MB), eta = 1e-3: 20 iterations against the dense oracle."""
    w = W.image_grid()
    C = np.asarray(w.C, np.float64)
    K = float(C.max())
    s, _, _ = gpu_solver(w, eta=w.eta, check_every=10)
    P = O.LampParams(eta=w.eta, K=K)
    done, ref = 0, None
    for T in (1, 5, 20):
        s.iterate(T - done)
        ref = O.lamp_run(C, w.r, w.c, P, T - done, state=ref)
        done = T
        assert_pot_close(s.get_state(), ref, what=f"image_grid T={T}")
    obj = s.objective()
    rep = O.objective_report(C, w.r, w.c, K, w.eta, ref)
    assert_logZ_close(s.get_state()["logZ"], rep["logZ"], what="image_grid log Z")
    assert abs(obj["cost"] - rep["cost"]) <= OBJ_TOL * rep["cost"]
    assert abs(obj["entropy"] - rep["entropy"]) <= 1e-6 * abs(rep["entropy"])
    s.close()


def test_diffloss_fullsize_gradient():
    """n = m = 8192, d = 3, eta = 1e-2: after 10 iterations the backward kernel's
    sum_j X_ij dC_ij/dx_i (and the y side) against the oracle's envelope formula on
    its own X^10; and translation invariance sum_i dx_i + sum_j dy_j = 0."""
    w = W.diffloss()
    C, sc, K = oracle_cost(w)
    T = 10
    s, _, _ = gpu_solver(w, eta=w.eta, check_every=10)
    s.iterate(T)
    dx, dy = s.grad()
    dx = dx.cpu().numpy().astype(np.float64)
    dy = dy.cpu().numpy().astype(np.float64)
    st = O.lamp_run(C, w.r, w.c, O.LampParams(eta=w.eta, K=K), T)
    X = w.r[:, None] * O.dual_to_primal(C, K, st.kappa, st.nu)[0]
    gx, gy = O.grad_envelope(w.x, w.y, X)
    del X, C
    assert np.abs(dx - gx).max() <= GRAD_TOL * np.abs(gx).max()
    assert np.abs(dy - gy).max() <= GRAD_TOL * np.abs(gy).max()
    tot = np.abs(dx).sum() + np.abs(dy).sum()
    assert np.abs(dx.sum(0) + dy.sum(0)).max() <= 1e-5 * tot
    s.close()


def test_plain_2d_full_solve_and_certificate():
    """n = m = 256, d = 2 (the FP64-checkable workload): solve to infeasibility 1e-6 on
    both sides; the certificate of Prop. infeas_bound (a) holds for the GPU's reported
    quantities against the exact OT value of the same cost (LP)."""
    w = W.plain_2d()
    C, sc, K = oracle_cost(w)
    tol = 1e-6
    s, _, _ = gpu_solver(w, tol=tol, max_iter=200000, check_every=100)
    res = s.solve(allow_not_converged=False)
    obj = s.objective()
    st, info, conv = O.lamp_solve(C, w.r, w.c, O.LampParams(K=K), tol, 200000)
    assert conv and res["converged"] and res["infeas"] <= tol
    ot = O.ot_lp(C, w.r, w.c)
    # the proof of Prop. infeas_bound (a) (App. D) bounds <C, X^t> - OT* <= 2K ||col - c||_1
    # + 2K log m / t, i.e. cost + 2K res <= OT* + certificate; and Round(X^t) is feasible
    # with ||X - Round(X)||_1 <= 2 res, so cost >= OT* - 2K res
    assert obj["cost"] + 2 * K * obj["col_res"] <= ot + obj["certificate"] + 1e-9
    assert obj["cost"] >= ot - 2 * K * obj["col_res"] - 1e-9
    assert abs(res["iters"] - st.t) <= max(2, 0.05 * st.t)
    s.close()
