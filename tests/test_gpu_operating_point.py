"""Parity where the headline results are decided, through the C ABI, against the FP64 oracle.

* Large kappa on the high-dimensional workload's own points: one iteration of Alg. 2 and one
  evaluation of X^{t+1} from the oracle's own states at t = 500 and t = 1170 (the headline
  solve's length at n = 2^15), on a 4096 x 4096 sample of the workload (the first 4096 source
  and target points).  The states come from tests/golden/highdim4096_states.npz, written by
  tests/golden/make_highdim_states.py with the oracle alone.
* The differentiable-loss workload at full size (n = m = 8192, d = 3, eta = 1e-2): the
  gradient at the target regularisation kappa = 1/eta against central finite differences
  in FP64.
* The large-scale recipe (U[0,1]^3, random marginals) at n = m = 2^14, where the direct-form
  sweeps run with split inner ranges over several waves as at 2^18: five iterations from
  the Alg. 2 start against the streamed oracle.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_util import (GRAD_TOL, LOGZ_TOL, OBJ_TOL, POT_TOL, RES_FLOOR, assert_logZ_close, assert_pot_close,
                            dev, gpu_solver, gpu_solver_raw, oracle_cost)

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "highdim4096_states.npz")


def _golden():
    z = np.load(GOLDEN)
    return {k: z[k] for k in z.files}


def _sample(variant):
    """The 4096 x 4096 sample of the highdim workload the golden states were computed on."""
    g = _golden()
    n = int(g["n"])
    w = W.highdim(seed=int(g["seed"]))
    x = np.ascontiguousarray(w.x[:n])
    y = np.ascontiguousarray(w.y[:n])
    xr, yr = (W.bf16_round(x), W.bf16_round(y)) if variant == "bf16" else (x, y)
    ws = W.Workload(name="highdim4096", kind="sqeuclid", n=n, m=n, d=w.d, r=W.uniform_marginal(n),
                    c=W.uniform_marginal(n), x=x, y=y, cost_scale=1.0, eta=0.0, tol=1e-6, seed=w.seed)
    return g, ws, O.sqeuclid_cost(xr, yr)


def _state(g, variant, key):
    return O.LampState(int(key) if key != "stop" else int(g[f"{variant}_t_stop"]), float(g[f"{variant}_kappa_{key}"]),
                       g[f"{variant}_nu_{key}"].copy(), g[f"{variant}_theta_{key}"].copy())


def _dot_slack(x, y, kappa):
    """Widening of the potential tolerance for the float32 accumulation of x.y (tensor cores
    or CUDA cores) at kappa.  The kernels see C~ = C + delta with delta_ij = -2 (z~_ij - z_ij),
    z~ the float32 accumulation of the d products; the exponents then differ by kappa
    |delta| and, like cost_slack in gpu_util, the potentials by up to 4 kappa max|delta|.
    delta is estimated by accumulating the products in float32 in coordinate order on the
    host (the kernels' order differs, so this is an estimate of the size, not of the sign)."""
    x32 = np.asarray(x, np.float32)
    y32 = np.asarray(y, np.float32)
    z32 = np.zeros((x32.shape[0], y32.shape[0]), np.float32)
    for k in range(x32.shape[1]):
        z32 += np.outer(x32[:, k], y32[:, k]).astype(np.float32)
    z64 = x32.astype(np.float64) @ y32.astype(np.float64).T
    return 4.0 * kappa * 2.0 * float(np.abs(z32.astype(np.float64) - z64).max())


@pytest.mark.parametrize("prec,T0", [("bf16_tc", 500), ("bf16_tc", 1170), ("fp32", 500), ("fp32", 1170)])
def test_step_and_evaluation_at_headline_kappa(prec, T0):
    """One iteration from the oracle's state t = T0 and the evaluation of X^{T0+1}: nu, theta,
    log Z against the oracle (bf16 tensor cores: on the rounded points, the problem that path
    solves; float32 dot form: on the points as given), <C, X> to 1e-6."""
    variant = "bf16" if prec == "bf16_tc" else "fp32"
    g, w, C = _sample(variant)
    K = float(g[f"{variant}_K"])
    assert K == O.sup_norm(C)
    st0 = _state(g, variant, str(T0))
    assert st0.t == T0 and st0.kappa == pytest.approx(T0 / (2 * K), rel=1e-12)
    sol = gpu_solver_raw(w, K, 1.0, prec=prec, check_every=1)
    sol.set_state(st0.nu, st0.theta, st0.kappa, st0.t)
    sol.iterate(1)
    ca = O.calpha_of(w.c, 0.01)
    ref1, info = O.lamp_step(C, w.r, w.c, K, 1 / (2 * K), 1 / (2 * K), 0.0, ca, 1.1, st0)
    got = sol.get_state()
    dnu = np.abs(got["nu"] - ref1.nu).max()
    dth = np.abs(got["theta"] - ref1.theta).max()
    # tensor cores: the products of bf16 points are exact and the MMA's float32 accumulation
    # keeps the potentials within the plain 1e-5 (measured 2.3e-6 at t = 500, 6.7e-6 at
    # t = 1170); the float32 dot form rounds every product and partial sum, so its potentials
    # move by up to ~kappa |delta| (measured 7.6e-6 at t = 500, 1.9e-5 at t = 1170)
    tol = POT_TOL if prec == "bf16_tc" else POT_TOL + _dot_slack(w.x, w.y, st0.kappa)
    print(f"\n{prec} T0={T0}: |dnu|={dnu:.3e} |dtheta|={dth:.3e} tol={tol:.3e} (plain {POT_TOL:.0e})")
    assert dnu <= tol and dth <= tol
    # evaluation of X^{T0+1} from the oracle's state (log Z and <C, X>)
    sol.set_state(ref1.nu, ref1.theta, ref1.kappa, ref1.t)
    obj = sol.objective()
    rep = O.objective_report(C, w.r, w.c, K, 0.0, ref1)
    lz = sol.get_state()["logZ"]
    lz_err = float((np.abs(lz - rep["logZ"]) / (1.0 + np.abs(rep["logZ"]))).max())
    cost_err = abs(obj["cost"] - rep["cost"]) / abs(rep["cost"])
    print(f"{prec} T0={T0}: logZ rel err {lz_err:.3e}, <C,X> rel err {cost_err:.3e}, "
          f"res gpu {obj['col_res']:.4e} oracle {rep['col_res']:.4e}")
    assert lz_err <= (LOGZ_TOL if prec == "bf16_tc" else LOGZ_TOL + tol)
    assert cost_err <= OBJ_TOL
    sol.close()


def _semi_dual_rows(Crows, K, kappa, nu, rsub):
    """F restricted to some rows: -(1/kappa) sum_i r_i log Z_i with log Z_i the oracle's
    row normaliser of exp(-kappa (C_ij + 2K nu_j)); X = diag(r) p^{1/kappa}(nu) is the exact
    minimiser of <C + 2K 1 nu^T, X> - H(X)/kappa over row-feasible X, so dF/dx_i =
    sum_j X_ij dC_ij/dx_i (and likewise for y_j)."""
    return -float(rsub @ O.log_normalizers(Crows, K, kappa, nu)) / kappa


def test_diffloss_gradient_matches_fd_at_target_kappa():
    """n = m = 8192, d = 3, eta = 1e-2 (the differentiable-loss workload): the state nu^10,
    theta^10 of the oracle with kappa = 1/eta (the target regularisation, where the
    exponents are sharpest).  lamp_grad against central FP64 finite differences of F (see
    _semi_dual_rows) on 64 fixed source points (every coordinate) and, for the target side,
    along three random directions supported on 64 fixed target points."""
    w = W.diffloss()
    C, sc, K = oracle_cost(w)
    eta = w.eta
    st = O.lamp_run(C, w.r, w.c, O.LampParams(eta=eta, K=K), 10)
    kap = 1.0 / eta
    s, _, _ = gpu_solver(w, eta=eta, check_every=10)
    s.set_state(st.nu, st.theta, kap, st.t)
    dx, dy = s.grad()
    dx = dx.cpu().numpy().astype(np.float64)
    dy = dy.cpu().numpy().astype(np.float64)
    s.close()
    x64 = w.x.astype(np.float64)
    y64 = w.y.astype(np.float64)
    rng = np.random.default_rng(404)
    rows = np.sort(rng.choice(w.n, 64, replace=False))
    h = 2e-6
    worst = 0.0
    for i in rows:
        for k in range(3):
            v = []
            for sg in (1.0, -1.0):
                xi = x64[i:i + 1].copy()
                xi[0, k] += sg * h
                v.append(_semi_dual_rows(O.sqeuclid_cost(xi, y64), K, kap, st.nu, w.r[i:i + 1]))
            fd = (v[0] - v[1]) / (2 * h)
            err = abs(dx[i, k] - fd) / max(abs(fd), 1e-2 * np.abs(dx).max())
            worst = max(worst, err)
    print(f"\nx side: worst relative error against FD {worst:.3e}")
    assert worst <= GRAD_TOL
    cols = np.sort(rng.choice(w.m, 64, replace=False))
    hy = 1e-5
    for rep in range(3):
        U = rng.standard_normal((64, 3))
        v = []
        for sg in (1.0, -1.0):
            yp = y64.copy()
            yp[cols] += sg * hy * U
            v.append(_semi_dual_rows(O.sqeuclid_cost(x64, yp), K, kap, st.nu, w.r))
        fd = (v[0] - v[1]) / (2 * hy)
        an = float((dy[cols] * U).sum())
        print(f"y direction {rep}: FD {fd:.9e} lamp_grad {an:.9e}")
        assert abs(an - fd) <= GRAD_TOL * abs(fd)


def _expanded_rows(x, y):
    x64 = np.asarray(x, np.float64)
    y64 = np.asarray(y, np.float64)
    return lambda rows: O.sqeuclid_cost(x64[rows], y64, chunk=len(rows))


def test_largescale_recipe_trajectory_at_2_14():
    """The large-scale recipe (U[0,1]^3 points, random marginals, eta = 0) at n = m = 2^14:
    the direct-form sweeps run 19 inner splits (ragged last split) over several waves, the
    path they take at 2^18.  Five iterations from the Alg. 2 start, all potentials and log Z
    of X^5 against the oracle streaming C in row blocks."""
    w = W.largescale(n=1 << 14)
    rows = _expanded_rows(w.x, w.y)
    K = O.streamed_sup_norm(rows, w.n, chunk=1024)
    P = O.LampParams(K=K)
    tau = 1.0 / (2.0 * K)
    ca = O.calpha_of(w.c, P.alpha)
    st = O.lamp_initial_state(w.m)
    T = 5
    for _ in range(T):
        st, _ = O.lamp_step_streamed(rows, w.n, w.r, w.c, K, tau, tau, 0.0, ca, P.beta, st, chunk=1024)
    colT, logZT = O.col_entries(rows, w.n, np.arange(w.m), K, st.kappa, st.nu, w.r, chunk=1024)
    s = gpu_solver_raw(w, K, 1.0, check_every=5)
    s.iterate(T)
    obj = s.objective()
    g = s.get_state()
    assert g["t"] == T
    assert_pot_close(g, st, what="largescale 2^14 T=5")
    assert_logZ_close(g["logZ"], logZT, what="largescale 2^14 log Z")
    res = float(np.abs(colT - w.c).sum())
    assert abs(obj["col_res"] - res) <= 1e-6 * res + RES_FLOOR
    s.close()


def test_precision_against_the_unrounded_problem():
    """The error each GPU precision makes against the FP64 oracle on the unrounded problem
    (the 4096 x 4096 sample; the oracle's state at its stop t = 1269 from the golden file),
    both paths run as a user runs them (K from their own cost) for the same t.
    Bounds stated here (measured values in parentheses):
      float32 dot form   potentials <= 2e-5 (3.1e-6), <C, X> <= 1e-7 relative (1.8e-9);
      bf16 tensor cores  potentials <= 2e-3 (3.7e-4), <C, X> <= 5e-5 relative (8.4e-6):
        the bf16 rounding of the points moves C by up to 0.55 (0.18 % of K) and the
        trajectory with it; the objective moves far less because the rounding errors
        average over the plan.
    Both paths reach infeasibility <= 1e-6 within 1 % of the oracle's iteration count."""
    import paper_2511_11359_gb300 as L

    g, w, C = _sample("fp32")
    T = int(g["fp32_t_stop"])
    nu_T, th_T, kap_T = g["fp32_nu_stop"], g["fp32_theta_stop"], float(g["fp32_kappa_stop"])
    K = float(g["fp32_K"])
    X = w.r[:, None] * O.dual_to_primal(C, K, kap_T, nu_T)[0]
    cost_T = float((C * X).sum())
    del X
    bounds = {"fp32": (2e-5, 1e-7), "bf16_tc": (2e-3, 5e-5)}
    for prec, (pot_b, cost_b) in bounds.items():
        s = L.Lamp(dev(w.r), dev(w.c), x=dev(w.x), y=dev(w.y), cost_scale=1.0, prec=prec, check_every=50)
        s.iterate(T)
        obj = s.objective()
        st = s.get_state()
        s.close()
        dpot = max(np.abs(st["nu"] - nu_T).max(), np.abs(st["theta"] - th_T).max())
        dcost = abs(obj["cost"] - cost_T) / cost_T
        print(f"\n{prec}: potentials {dpot:.3e}, <C,X> rel {dcost:.3e}")
        assert dpot <= pot_b and dcost <= cost_b
        s = L.Lamp(dev(w.r), dev(w.c), x=dev(w.x), y=dev(w.y), cost_scale=1.0, prec=prec, tol=1e-6, check_every=50)
        res = s.solve(allow_not_converged=False)
        s.close()
        assert abs(res["iters"] - T) <= 0.01 * T, res["iters"]
