"""The bf16 tcgen05 path (LAMP_PREC_BF16_TC) against the FP64 oracle run on the
bf16-rounded points (the problem that path solves), through the C ABI."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_util import (POT_TOL, RES_FLOOR, assert_logZ_close, assert_pot_close, gpu_solver, gpu_solver_raw,
                            oracle_cost)

pytestmark = pytest.mark.gpu


def rounded(w):
    """The workload with its points rounded to bf16 (what the tensor cores multiply)."""
    return dataclasses.replace(w, x=W.bf16_round(w.x), y=W.bf16_round(w.y))


def test_bf16_round_helper():
    a = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 1e-3], np.float32)
    r = W.bf16_round(a)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125  # ties to even, then round up
    assert np.all(np.abs(r - a) <= np.abs(a) * 2.0 ** -8)


TC_CASES = [
    ("hd64", 300, 257, 64, "gauss_shift", "uniform", 1.0, 0.0),
    ("hd17", 129, 300, 17, "gauss_shift", "random", 0.05, 0.0),
    ("d3eta", 200, 200, 3, "sphere", "uniform", 1.0, 1e-2),
    ("ragged", 1, 130, 64, "gauss_shift", "random", 1.0, 0.0),
    ("ragged2", 257, 1, 33, "uniform", "random", 1.0, 0.0),
]


@pytest.mark.parametrize("case", TC_CASES, ids=[c[0] for c in TC_CASES])
def test_tc_trajectory_matches_oracle_on_rounded_points(case):
    name, n, m, d, dist, marg, scale, eta = case
    w = W.points_problem(name, n, m, d, seed=sum(name.encode()) % 997, dist=dist, marg=marg, cost_scale=scale, eta=eta)
    wr = rounded(w)
    C, s, K = oracle_cost(wr)
    # the GPU is given the unrounded points and rounds them itself
    sol, _, _ = gpu_solver(w, K=K, scale=s, eta=eta, prec="bf16_tc", check_every=6)
    P = O.LampParams(eta=eta, K=K)
    done, ref = 0, None
    for T in (1, 10, 100):
        sol.iterate(T - done)
        ref = O.lamp_run(C, wr.r, wr.c, P, T - done, state=ref)
        done = T
        assert_pot_close(sol.get_state(), ref, what=f"{name} T={T}")
    obj = sol.objective()
    rep = O.objective_report(C, wr.r, wr.c, K, eta, ref)
    assert abs(obj["cost"] - rep["cost"]) <= 1e-6 * abs(rep["cost"])
    assert_logZ_close(sol.get_state()["logZ"], rep["logZ"], what=f"{name} logZ")
    sol.close()


@pytest.mark.parametrize("T0", [500, 3000])
def test_tc_single_step_at_large_kappa_exact_cost(T0):
    """Dyadic coordinates k/16 (|k| < 256) are exact in bf16 and every x.y is exact in
    float32, so the tensor-core cost equals the oracle's: tolerance 1e-5."""
    w = W.points_problem("lk", 96, 130, 16, seed=7, dist="gauss_shift", cost_scale=1.0, grid_step=16)
    assert np.array_equal(W.bf16_round(w.x), w.x) and np.array_equal(W.bf16_round(w.y), w.y)
    s, C, K = gpu_solver(w, prec="bf16_tc", check_every=1)
    P = O.LampParams(K=K)
    st0 = O.lamp_run(C, w.r, w.c, P, T0)
    s.set_state(st0.nu, st0.theta, st0.kappa, st0.t)
    s.iterate(1)
    K_, tau1, tau2 = O.resolve_params(C, P)
    ref1, info = O.lamp_step(C, w.r, w.c, K_, tau1, tau2, 0.0, O.calpha_of(w.c, 0.01), 1.1, st0)
    assert_pot_close(s.get_state(), ref1, tol=POT_TOL, what=f"tc step at t={T0}")
    s.close()


def test_tc_solve_reaches_tolerance_like_fp32():
    """Both precisions reach infeasibility <= 1e-6 on the same problem; the bf16 path's
    answer is the optimum of the rounded problem (its cost within 1e-3 of the fp32 one)."""
    w = W.highdim(n=1024, seed=5)
    res = {}
    for prec in ("fp32", "bf16_tc"):
        s, C, K = gpu_solver(w, prec=prec, tol=1e-6, max_iter=100000, check_every=100)
        r = s.solve(allow_not_converged=False)
        res[prec] = (r, s.objective())
        s.close()
    assert res["fp32"][0]["infeas"] <= 1e-6 and res["bf16_tc"][0]["infeas"] <= 1e-6
    c32, c16 = res["fp32"][1]["cost"], res["bf16_tc"][1]["cost"]
    assert abs(c16 - c32) <= 1e-3 * abs(c32)


def test_tc_checkpoint_resume_bitwise():
    w = W.highdim(n=300, seed=9)
    a, C, K = gpu_solver(w, prec="bf16_tc", check_every=4)
    a.iterate(21)
    ck = a.get_state()
    a.iterate(13)
    ea = a.get_state()
    b, _, _ = gpu_solver(w, prec="bf16_tc", check_every=7)
    b.set_state(ck["nu"], ck["theta"], ck["kappa"], ck["t"], ck["row_shifts"])
    b.iterate(13)
    eb = b.get_state()
    assert np.array_equal(ea["nu"], eb["nu"]) and np.array_equal(ea["theta"], eb["theta"])
    a.close()
    b.close()


def test_tc_iteration_matches_oracle_at_4096():
    """Many tiles per CTA and a full grid: one bf16 iteration from the same oracle state
    and the evaluation of log Z, against the oracle on the rounded points."""
    w = W.highdim(n=4096, seed=13)
    wr = rounded(w)
    C, s, K = oracle_cost(wr)
    P = O.LampParams(K=K)
    st0 = O.lamp_run(C, wr.r, wr.c, P, 3)
    sol, _, _ = gpu_solver(w, K=K, scale=s, prec="bf16_tc", check_every=1)
    sol.set_state(st0.nu, st0.theta, st0.kappa, st0.t)
    sol.iterate(1)
    K_, tau1, tau2 = O.resolve_params(C, P)
    ref1, info = O.lamp_step(C, wr.r, wr.c, K_, tau1, tau2, 0.0, O.calpha_of(wr.c, 0.01), 1.1, st0)
    assert_pot_close(sol.get_state(), ref1, what="tc 4096 step")
    sol.set_state(ref1.nu, ref1.theta, ref1.kappa, ref1.t)
    obj = sol.objective()
    rep = O.objective_report(C, wr.r, wr.c, K, 0.0, ref1)
    assert_logZ_close(sol.get_state()["logZ"], rep["logZ"], what="tc 4096 logZ")
    assert abs(obj["cost"] - rep["cost"]) <= 1e-6 * abs(rep["cost"])
    sol.close()


def test_tc_solve_4096_converges_like_fp32():
    """At a size with many tiles per CTA both precisions reach 1e-6 in about the same
    number of iterations (they solve nearly the same problem)."""
    w = W.highdim(n=4096, seed=3)
    its = {}
    for prec in ("fp32", "bf16_tc"):
        s, C, K = gpu_solver(w, prec=prec, tol=1e-6, max_iter=20000, check_every=50)
        r = s.solve(allow_not_converged=False)
        its[prec] = r["iters"]
        s.close()
    assert abs(its["bf16_tc"] - its["fp32"]) <= 0.1 * its["fp32"], its


@pytest.mark.parametrize("n,iters", [(8192, 400), (1 << 15, 600)])
def test_tc_run_is_deterministic_across_graph_lengths(n, iters):
    """The same bf16 problem iterated with different device-loop lengths gives bit-identical
    potentials and row shifts (no race in the pipelined kernels).  n = 2^15, d = 64 is the
    full-size highdim workload: 74 streamed tiles per CTA, three waves of CTAs; a
    write-after-read race between the epilogue's reads of a packed-pair buffer and the
    next bulk copy into it once changed ~10 % of its iterations."""
    w = W.highdim(n=n, seed=21)
    out = []
    for ce in (50, 7):
        s = gpu_solver_raw(w, None, prec="bf16_tc", check_every=ce)  # K from the device pass
        s.iterate(iters)
        out.append(s.get_state())
        s.close()
    for key in ("nu", "theta", "row_shifts"):
        assert np.array_equal(out[0][key], out[1][key]), key


@pytest.mark.parametrize("n,m,d", [(300, 257, 17), (1000, 999, 64), (4096, 3000, 64)])
def test_tc_k_pass_matches_the_rounded_cost(n, m, d):
    """A tensor-core context takes K = max C from its own sweep (D = |x|^2 + |y|^2 - 2 x.y over
    the MMA's products of the bf16 points, columns past m skipped): K matches the maximum
    of the oracle's cost on the rounded points to float32 rounding."""
    import torch
    import paper_2511_11359_gb300 as L

    w = W.highdim(n=n, m=m, d=d, seed=n + m)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    with L.Lamp(t(w.r), t(w.c), x=t(w.x), y=t(w.y), prec="bf16_tc") as s:
        K = s.objective()["K"]
    Kref = float(O.sqeuclid_cost(W.bf16_round(w.x), W.bf16_round(w.y)).max())
    assert abs(K - Kref) <= 1e-6 * Kref, (K, Kref)
