"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms, the PDMP / Alg. 4 equivalences, a numeric argmax of the dual
mirror-map objective, exact OT (LP and permutation brute force), FP64 Sinkhorn,
Round's guarantees and the invariants the paper proves.

All CPU-only (not marked gpu)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def small_points(n, m, d=2, seed=0, marg="random", scale=-1.0):
    w = W.points_problem("t", n, m, d, seed, dist="uniform", marg=marg, cost_scale=scale)
    return O.cost_matrix(w), w.r, w.c


# ----------------------------------------------------------------------------- kappa


@pytest.mark.parametrize("eta", [0.0, 1e-3, 0.05, 0.7])
def test_kappa_recursion_matches_closed_form(eta):
    """Section 3.2: 1/eta_{t+1} = (1 - (1 - tau1 eta)^{t+1})/eta and tau1 t at eta=0."""
    tau1 = 0.37
    kap = 0.0
    for t in range(1, 400):
        kap = O.kappa_next(kap, eta, tau1)
        if eta == 0.0:
            ref = tau1 * t
        else:
            ref = (1.0 - (1.0 - tau1 * eta) ** t) / eta
        assert abs(kap - ref) <= 1e-12 * max(1.0, ref)
    # eta_1 = 1/tau1 from the eta_0 -> infinity limit
    assert O.kappa_next(0.0, eta, tau1) == tau1


def test_kappa_limit_is_one_over_eta():
    tau1, eta = 0.5, 0.2
    kap = 0.0
    for _ in range(2000):
        kap = O.kappa_next(kap, eta, tau1)
    assert abs(kap - 1.0 / eta) < 1e-12


# ----------------------------------------------------------------------------- start


@pytest.mark.parametrize("n,m", [(5, 9), (33, 17)])
def test_uniform_start(n, m):
    """Proof of Prop. equivalence, base case: p^{eta_0}(nu^0) = 1/m, so col(X^0) = 1/m exactly."""
    C, r, c = small_points(n, m, seed=3)
    rec = []
    O.lamp_run(C, r, c, O.LampParams(), 1, record=lambda s, i: rec.append(i))
    A = rec[0].A
    assert np.max(np.abs(A - 1.0 / m)) < 1e-15
    assert abs(rec[0].res - np.abs(1.0 / m - c).sum()) < 1e-14


# ----------------------------------------------------------------------------- LAMP == PDMP


@pytest.mark.parametrize("eta", [0.0, 1e-2])
@pytest.mark.parametrize("n,m,seed", [(7, 5, 1), (16, 16, 2), (40, 64, 3)])
def test_lamp_equals_explicit_pdmp(n, m, seed, eta):
    """Prop. equivalence: p^t = p^{eta_t}(nu^t) and pbar^{t+1} = p^{eta_{t+1}}(nubar^{t+1}),
    with PDMP run with explicit O(nm) primal iterates (Alg. 1)."""
    C, r, c = small_points(n, m, seed=seed)
    P = O.LampParams(eta=eta)
    K, tau1, tau2 = O.resolve_params(C, P)
    T = 60
    pd = []
    O.pdmp_run(C, r, c, P, T, record=lambda t, p, pbar, th: pd.append((p.copy(), pbar.copy(), th.copy())))
    la = []

    def rec(s, info):
        p_t, _ = O.dual_to_primal(C, K, s.kappa, s.nu)
        pbar, _ = O.dual_to_primal(C, K, info.kappa_next, info.nubar)
        la.append((p_t, pbar, s.theta.copy()))

    O.lamp_run(C, r, c, P, T, record=rec)
    for t in range(T):
        assert np.max(np.abs(pd[t][0] - la[t][0])) < 1e-12, t
        assert np.max(np.abs(pd[t][1] - la[t][1])) < 1e-12, t
        assert np.max(np.abs(pd[t][2] - la[t][2])) < 1e-12, t


def test_alg2_equals_alg4_performant():
    """App. D: with eta = 0, tau1 = tau2 = 1/(2K), beta = log 3, Alg. 2 is Alg. 4."""
    C, r, c = small_points(20, 30, seed=5, scale=3.7)  # unnormalised cost (K != 1)
    T = 200
    nu4, th4 = O.lamp_performant_run(C, r, c, 0.01, T)
    st = O.lamp_run(C, r, c, O.LampParams(eta=0.0, beta=math.log(3.0)), T)
    assert np.max(np.abs(st.nu - nu4)) < 1e-11
    assert np.max(np.abs(st.theta - th4)) < 1e-11


# ----------------------------------------------------------------------------- dual step


def test_dual_mirror_map_is_the_argmax():
    """Eq. def:closed_form_opt (second line) against a numeric 1-D maximisation of
    tau <grad G, theta> - D_{H_c^alpha}(theta || theta0), with the Bregman divergence
    written from the definition of H_c^alpha (Section 3.1), not from the oracle."""
    from scipy.optimize import minimize_scalar

    rng = np.random.default_rng(7)
    m = 12
    c = rng.uniform(0.1, 1.0, m)
    c /= c.sum()
    alpha, tau, K = 0.01, 0.3, 2.5
    ca = c + alpha / m
    theta0 = rng.uniform(-0.6, 0.6, m)
    colr = c + rng.normal(0.0, 0.05, m)

    def H(v, a):
        return a * ((1 + v) / 2 * np.log((1 + v) / 2) + (1 - v) / 2 * np.log((1 - v) / 2))

    def dH(v, a):
        return a * 0.5 * np.log((1 + v) / (1 - v))

    closed = O.dual_mirror_map(theta0, colr, c, ca, tau, K)
    for j in range(m):
        g = 2.0 * K * (colr[j] - c[j])

        def negobj(th):
            breg = H(th, ca[j]) - H(theta0[j], ca[j]) - dH(theta0[j], ca[j]) * (th - theta0[j])
            return -(tau * g * th - breg)

        res = minimize_scalar(negobj, bounds=(-1 + 1e-12, 1 - 1e-12), method="bounded",
                              options={"xatol": 1e-13})
        assert abs(res.x - closed[j]) < 1e-7


def test_tclip_bounds():
    th = np.linspace(-0.99, 0.99, 101)
    b = math.tanh(1.1 / 2)
    out = O.tclip(th, 1.1)
    assert out.max() == pytest.approx(b) and out.min() == pytest.approx(-b)
    assert np.all(out[np.abs(th) <= b] == th[np.abs(th) <= b])
    # log 3 gives exactly the [-1/2, 1/2] box of Alg. 4
    assert math.tanh(math.log(3.0) / 2) == pytest.approx(0.5, abs=1e-15)


# ----------------------------------------------------------------------------- entropy identity


@pytest.mark.parametrize("eta", [0.0, 0.05])
def test_entropy_identity(eta):
    """Lemma pd_obj_relation (App. D), general kappa: H(X) from log Z, <C,X>, col(X), nu."""
    C, r, c = small_points(25, 31, seed=9)
    P = O.LampParams(eta=eta)
    K, _, _ = O.resolve_params(C, P)
    st = O.lamp_initial_state(31)
    for T in [0, 1, 5, 50, 300]:
        st_T = O.lamp_run(C, r, c, P, T)
        p, logZ = O.dual_to_primal(C, K, st_T.kappa, st_T.nu)
        X = r[:, None] * p
        H_dense = O.entropy(X)
        H_id = O.entropy_from_normalizers(r, logZ, st_T.kappa, K, float((C * X).sum()), X.sum(0), st_T.nu)
        assert abs(H_dense - H_id) < 1e-10 * max(1.0, abs(H_dense))
    # eta_0 = infinity start: X^0 = diag(r)/m, H(X^0) = H(r) + log m
    Hr = -(r * np.log(r)).sum()
    X0 = r[:, None] * np.full((25, 31), 1 / 31)
    assert abs(O.entropy(X0) - (Hr + math.log(31))) < 1e-12


# ----------------------------------------------------------------------------- exact OT


@pytest.mark.parametrize("n", [3, 5, 7])
def test_lp_matches_permutation_bruteforce(n):
    """Birkhoff: for uniform marginals on n = m points an optimal plan is a permutation."""
    rng = np.random.default_rng(100 + n)
    C = rng.uniform(0, 1, (n, n))
    u = np.full(n, 1.0 / n)
    assert abs(O.ot_lp(C, u, u) - O.ot_bruteforce_uniform(C)) < 1e-9


def test_lp_trivial_cases():
    # zero cost on the diagonal of a 1-1 problem; rank-one cost
    C = np.array([[0.0, 1.0], [1.0, 0.0]])
    u = np.array([0.5, 0.5])
    assert abs(O.ot_lp(C, u, u)) < 1e-12
    a = np.array([0.2, 0.3, 0.5])
    b = np.array([0.6, 0.4])
    Crank = np.add.outer(np.array([1.0, 2.0, 3.0]), np.array([0.5, 4.0]))  # separable: every plan costs the same
    assert abs(O.ot_lp(Crank, a, b) - (a @ [1, 2, 3] + b @ [0.5, 4.0])) < 1e-9


@pytest.mark.parametrize("beta", [1.1, math.log(3.0)])
def test_eta0_certificate_and_weak_duality(beta):
    """Prop. infeas_bound (a) at every t: <C, Round(X^t)> - OT* <= 4K res_t + 2K log m / t;
    weak duality D(theta) <= OT* <= <C, Round(X^t)> (App. B, Lemma jason_rounding);
    and the rounded cost approaches OT*."""
    n, m = 10, 12
    C, r, c = small_points(n, m, seed=21, scale=2.0)
    K = O.sup_norm(C)
    ot = O.ot_lp(C, r, c)
    P = O.LampParams(eta=0.0, beta=beta)
    gaps = []

    def rec(s, info):
        if s.t == 0:
            return
        X = r[:, None] * O.dual_to_primal(C, K, s.kappa, s.nu)[0]
        Xr = O.round_plan(X, r, c)
        rc = float((C * Xr).sum())
        col_res = float(np.abs(X.sum(0) - c).sum())
        assert rc - ot <= O.certificate_rhs(K, col_res, m, s.t) + 1e-12
        assert rc >= ot - 1e-10
        assert O.saddle_dual(C, r, c, K, s.theta) <= ot + 1e-12
        assert O.saddle_dual(C, r, c, K, s.nu) <= ot + 1e-12
        gaps.append(rc - ot)

    O.lamp_run(C, r, c, P, 3000, record=rec)
    assert gaps[-1] < 1e-4 * max(ot, 1e-3)


def _lp_potentials(C, r, c):
    """Optimal LP potentials (u, v) with u_i + v_j <= C_ij and <r,u> + <c,v> = OT*,
    taken from the HiGHS dual values of the equality constraints."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix, vstack

    n, m = C.shape
    idx = np.arange(n * m)
    A = vstack([coo_matrix((np.ones(n * m), (idx // m, idx)), shape=(n, n * m)),
                coo_matrix((np.ones(n * m), (idx % m, idx)), shape=(m, n * m))]).tocsr()
    res = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([r, c]), bounds=(0, None), method="highs")
    y = res.eqlin.marginals
    return res.fun, y[:n], y[n:]


def test_saddle_dual_strong_duality_at_lp_potentials():
    """App. B / Lemma b_choice: with theta* = -v*/(2K) from optimal LP potentials,
    D(theta*) = OT* (the row constraint is kept, the column one is dualised)."""
    C, r, c = small_points(9, 11, seed=23, scale=1.5)
    K = O.sup_norm(C)
    ot, u, v = _lp_potentials(C, r, c)
    assert np.max(u[:, None] + v[None, :] - C) < 1e-9
    assert abs(r @ u + c @ v - ot) < 1e-9
    assert abs(O.saddle_dual(C, r, c, K, -v / (2 * K)) - ot) < 1e-9
    # and any other theta gives a lower bound
    rng = np.random.default_rng(0)
    for _ in range(5):
        assert O.saddle_dual(C, r, c, K, rng.uniform(-1, 1, 11)) <= ot + 1e-12


def test_entropic_saddle_dual_equals_eot_value_at_lamp_limit():
    """Strong duality for the eta > 0 saddle problem: at LAMP's limit (col(X) = c),
    D^eta(nu) = <C,X> - eta H(X), the EOT optimum.  This fixes the constant -eta H(r)."""
    n, m = 12, 15
    C, r, c = small_points(n, m, seed=43)
    K = O.sup_norm(C)
    eta = 0.05
    st, info, conv = O.lamp_solve(C, r, c, O.LampParams(eta=eta), tol=1e-13, max_iter=100000)
    assert conv
    X = r[:, None] * O.dual_to_primal(C, K, st.kappa, st.nu)[0]
    assert abs(O.saddle_dual(C, r, c, K, st.nu, eta) - O.eot_value(C, X, eta)) < 1e-9


def test_certificate_log_term_is_one_over_t():
    K, m = 1.7, 50
    vals = [O.certificate_rhs(K, 0.0, m, t) * t for t in (1, 2, 10, 1000)]
    assert np.allclose(vals, 2 * K * math.log(m), rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------- eta > 0 == Sinkhorn


def test_sinkhorn_pinned_to_lp():
    """Sinkhorn's plan is feasible and its cost lies in [OT*, OT* + eta log(nm)]."""
    C, r, c = small_points(14, 11, seed=31)
    ot = O.ot_lp(C, r, c)
    for eta in (0.1, 0.02, 0.005):
        X, f, g, _ = O.sinkhorn_log(C, r, c, eta, tol=1e-13)
        assert np.abs(X.sum(1) - r).sum() < 1e-12 and np.abs(X.sum(0) - c).sum() < 1e-12
        cx = float((C * X).sum())
        assert ot - 1e-10 <= cx <= ot + eta * math.log(14 * 11) + 1e-10


def test_lamp_eta_positive_converges_to_eot_optimum():
    """Lemma l1_prob_equiv (b): for eta <= K/log(max_j 1/c_j) the penalised problem and
    the EOT problem share their minimiser, so LAMP's limit is Sinkhorn's plan;
    potentials agree up to an additive constant (g = -2K nu + const)."""
    n, m = 18, 24
    C, r, c = small_points(n, m, seed=41)
    K = O.sup_norm(C)
    eta = 0.05
    assert eta <= K / math.log(1.0 / c.min())
    st, info, conv = O.lamp_solve(C, r, c, O.LampParams(eta=eta), tol=1e-13, max_iter=100000)
    assert conv
    X = r[:, None] * O.dual_to_primal(C, K, st.kappa, st.nu)[0]
    Xs, f, g, _ = O.sinkhorn_log(C, r, c, eta, tol=1e-14)
    assert abs(float((C * X).sum()) - float((C * Xs).sum())) <= 1e-9 * float((C * Xs).sum())
    assert np.max(np.abs(X - Xs)) < 1e-9
    gc = g - g.mean()
    nc = -2.0 * K * (st.nu - st.nu.mean())
    assert np.max(np.abs(gc - nc)) < 1e-7
    # the entropic objective of LAMP's plan equals the EOT optimum
    assert abs(O.eot_value(C, X, eta) - O.eot_value(C, Xs, eta)) < 1e-9


# ----------------------------------------------------------------------------- Round


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_round_is_feasible_and_within_bound(seed):
    """Lemma jason_rounding: Round(X) in Pi(r,c) and ||X - Round(X)||_1 <= 2(||row-r||_1 + ||col-c||_1)."""
    rng = np.random.default_rng(seed)
    n, m = 9, 13
    X = rng.uniform(0, 1, (n, m))
    X /= X.sum()
    r = rng.uniform(0.1, 1, n); r /= r.sum()
    c = rng.uniform(0.1, 1, m); c /= c.sum()
    Xr = O.round_plan(X, r, c)
    assert np.all(Xr >= -1e-16)
    assert np.abs(Xr.sum(1) - r).sum() < 1e-14 and np.abs(Xr.sum(0) - c).sum() < 1e-14
    bound = 2 * (np.abs(X.sum(1) - r).sum() + np.abs(X.sum(0) - c).sum())
    assert np.abs(X - Xr).sum() <= bound + 1e-14


def test_round_of_feasible_plan_is_identity():
    r = np.array([0.3, 0.7]); c = np.array([0.5, 0.5])
    X = np.outer(r, c)
    assert np.max(np.abs(O.round_plan(X, r, c) - X)) < 1e-16


# ----------------------------------------------------------------------------- invariants


def test_invariants_along_trajectory():
    """X >= 0, row(X^t) = r (Eq. row_feasible), sum_j col_j = 1, sum r = sum c = 1,
    theta and nu stay in (-1, 1) and the clip bound holds."""
    C, r, c = small_points(30, 20, seed=51)
    assert abs(r.sum() - 1) < 1e-15 and abs(c.sum() - 1) < 1e-15
    K = O.sup_norm(C)
    b = math.tanh(0.55)

    def rec(s, info):
        X = r[:, None] * O.dual_to_primal(C, K, s.kappa, s.nu)[0]
        assert X.min() >= 0.0
        assert np.abs(X.sum(1) - r).max() < 1e-15
        assert abs(info.A.sum() - 1.0) < 1e-14 and abs(info.B.sum() - 1.0) < 1e-14
        assert np.all(np.abs(s.theta) <= b + 1e-16)
        assert np.all(np.abs(s.nu) < 1.0)

    O.lamp_run(C, r, c, O.LampParams(), 400, record=rec)


def test_running_min_of_certificate_nonincreasing():
    C, r, c = small_points(12, 12, seed=61)
    K = O.sup_norm(C)
    vals = []
    O.lamp_run(C, r, c, O.LampParams(), 500,
               record=lambda s, i: vals.append(O.certificate_rhs(K, float(np.abs(i.A - c).sum()), 12, s.t)) if s.t else None)
    run = np.minimum.accumulate(vals)
    assert np.all(np.diff(run) <= 0)
    assert run[-1] < run[0]


def test_lamp_solve_stops_at_first_feasible_iterate():
    C, r, c = small_points(16, 16, seed=71)
    tol = 1e-5
    st, info, conv = O.lamp_solve(C, r, c, O.LampParams(), tol, 50000)
    assert conv and info.res <= tol
    # the previous iterate was not yet within tol
    rec = []
    O.lamp_run(C, r, c, O.LampParams(), st.t, record=lambda s, i: rec.append(i.res))
    assert min(rec) > tol


# ----------------------------------------------------------------------------- gradient


def test_envelope_gradient_matches_fd_of_sinkhorn_value():
    """dL/dx_i = sum_j X_ij dC_ij/dx_i for L = min_X <C,X> - eta H(X) (envelope theorem),
    against central finite differences of the FP64 Sinkhorn value, warm-started."""
    w = W.points_problem("g", 24, 20, 3, 5, dist="sphere", marg="uniform")
    x = w.x.astype(np.float64)
    y = w.y.astype(np.float64)
    eta = 0.05
    C = O.sqeuclid_cost(x, y)
    X, f, g, _ = O.sinkhorn_log(C, w.r, w.c, eta, tol=1e-14)
    dx, dy = O.grad_envelope(x, y, X)
    h = 1e-5
    for (i, k) in [(0, 0), (3, 2), (17, 1)]:
        vals = []
        for s in (+1, -1):
            xp = x.copy(); xp[i, k] += s * h
            Cp = O.sqeuclid_cost(xp, y)
            Xp, *_ = O.sinkhorn_log(Cp, w.r, w.c, eta, tol=1e-14, f0=f, g0=g)
            vals.append(O.eot_value(Cp, Xp, eta))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dx[i, k]) <= 1e-6 * max(1.0, abs(dx[i, k]))
    for (j, k) in [(1, 0), (19, 2)]:
        vals = []
        for s in (+1, -1):
            yp = y.copy(); yp[j, k] += s * h
            Cp = O.sqeuclid_cost(x, yp)
            Xp, *_ = O.sinkhorn_log(Cp, w.r, w.c, eta, tol=1e-14, f0=f, g0=g)
            vals.append(O.eot_value(Cp, Xp, eta))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dy[j, k]) <= 1e-6 * max(1.0, abs(dy[j, k]))


# ----------------------------------------------------------------------------- sampled evaluators


def test_sampled_evaluators_match_dense():
    C, r, c = small_points(50, 40, seed=81)
    K = O.sup_norm(C)
    st = O.lamp_run(C, r, c, O.LampParams(), 120)
    colX, logZ = O.marginals_from_state(C, r, K, st.kappa, st.nu)
    cols = np.array([0, 7, 39])
    cs, lz = O.col_entries(lambda rows: C[rows], 50, cols, K, st.kappa, st.nu, r, chunk=13)
    assert np.max(np.abs(cs - colX[cols])) < 1e-15
    assert np.max(np.abs(lz - logZ)) < 1e-12
    rows = np.array([2, 49])
    assert np.max(np.abs(O.logZ_rows(lambda rr: C[rr], rows, K, st.kappa, st.nu) - logZ[rows])) < 1e-12


def test_sqeuclid_cost_expansion_agrees():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((17, 5)); y = rng.standard_normal((23, 5))
    C = O.sqeuclid_cost(x, y, chunk=4)
    ref = (x ** 2).sum(1)[:, None] + (y ** 2).sum(1)[None, :] - 2 * x @ y.T
    assert np.max(np.abs(C - ref)) < 1e-12


def test_solve_does_not_stop_at_the_feasible_start():
    """Uniform c makes X^0 = diag(r)/m exactly feasible; the rule starts at t = 1."""
    w = W.points_problem("u", 12, 12, 2, 4, marg="uniform", cost_scale=1.0)
    C = O.cost_matrix(w)
    st, info, conv = O.lamp_solve(C, w.r, w.c, O.LampParams(), 1e-6, 20000)
    assert conv and st.t >= 1
    K = O.sup_norm(C)
    X0 = w.r[:, None] * O.dual_to_primal(C, K, 0.0, np.zeros(12))[0]
    assert np.abs(X0.sum(0) - w.c).sum() < 1e-15


def test_solve_eta_positive_waits_for_kappa():
    """For eta > 0 the rule also needs 1 - kappa_t eta <= tol (X^t solves the eta_t problem)."""
    C, r, c = small_points(10, 10, seed=3)
    eta, tol = 0.05, 1e-6
    st, info, conv = O.lamp_solve(C, r, c, O.LampParams(eta=eta), tol, 200000)
    assert conv and 1.0 - st.kappa * eta <= tol and info.res <= tol


def test_expanded_cost_matches_differences():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((40, 64)).astype(np.float32)
    y = (rng.standard_normal((33, 64)) + 0.5).astype(np.float32)
    assert np.max(np.abs(O.sqeuclid_cost_expanded(x, y) - O.sqeuclid_cost(x, y))) < 1e-10


def test_streamed_step_equals_dense_step():
    """lamp_step_streamed (row blocks of C) reproduces lamp_step (dense C)."""
    C, r, c = small_points(70, 45, seed=19)
    P = O.LampParams()
    K, tau1, tau2 = O.resolve_params(C, P)
    ca = O.calpha_of(c, P.alpha)
    st = O.lamp_run(C, r, c, P, 37)
    ref, info = O.lamp_step(C, r, c, K, tau1, tau2, 0.0, ca, P.beta, st)
    got, (A, B, lzA, lzB) = O.lamp_step_streamed(lambda rows: C[rows], 70, r, c, K, tau1, tau2, 0.0, ca, P.beta, st,
                                                chunk=16)
    assert np.max(np.abs(got.nu - ref.nu)) < 1e-13 and np.max(np.abs(got.theta - ref.theta)) < 1e-12
    assert np.max(np.abs(A - info.A)) < 1e-15 and np.max(np.abs(lzB - info.logZ_B)) < 1e-12
    assert O.streamed_sup_norm(lambda rows: C[rows], 70, chunk=9) == K


def test_point_costs_match_scipy_distances():
    """l1, l-inf and cosine ground costs (App. E.2) against scipy's cdist metrics
    'cityblock', 'chebyshev' and 'cosine' (1 - cos), an independent implementation."""
    from scipy.spatial.distance import cdist

    rng = np.random.default_rng(71)
    for d in (1, 3, 17):
        x = rng.normal(size=(23, d))
        y = rng.normal(size=(19, d)) + 0.3
        np.testing.assert_allclose(O.l1_cost(x, y), cdist(x, y, "cityblock"), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(O.linf_cost(x, y), cdist(x, y, "chebyshev"), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(O.cosine_cost(x, y), cdist(x, y, "cosine"), rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(O.l1_cost(x, y, 0.25), 0.25 * cdist(x, y, "cityblock"), rtol=1e-13)
    # cosine = half the squared distance of the unit-normalised points
    u = x / np.linalg.norm(x, axis=1, keepdims=True)
    v = y / np.linalg.norm(y, axis=1, keepdims=True)
    np.testing.assert_allclose(O.cosine_cost(x, y), 0.5 * O.sqeuclid_cost(u, v), rtol=1e-12, atol=1e-13)


# ----------------------------------------------------------------------------- exact penalty


def _lp_plan(C, r, c):
    """An optimal plan of Eq. prob:primal_ot from HiGHS (for the equality check below)."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix, vstack

    n, m = C.shape
    idx = np.arange(n * m)
    A = vstack([coo_matrix((np.ones(n * m), (idx // m, idx)), shape=(n, n * m)),
                coo_matrix((np.ones(n * m), (idx % m, idx)), shape=(m, n * m))]).tocsr()
    res = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([r, c]), bounds=(0, None), method="highs",
                  options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    return res.x.reshape(n, m)


def _row_feasible_family(C, r, Xstar, rng):
    """Row-feasible plans diag(r) p, p row-stochastic: Dirichlet rows, the greedy plan that
    puts each row's mass on its cheapest column (cost below OT*, large column residual),
    and blends of the greedy plan and of random plans with the optimum."""
    n, m = C.shape
    greedy = np.zeros((n, m))
    greedy[np.arange(n), C.argmin(axis=1)] = r
    fam = [greedy]
    for a in (0.05, 0.2, 0.5, 0.9):
        fam.append((1 - a) * Xstar + a * greedy)
    for conc in (0.05, 1.0, 20.0):
        p = rng.dirichlet(np.full(m, conc), size=n)
        fam.append(r[:, None] * p)
        fam.append(0.7 * Xstar + 0.3 * r[:, None] * p)
    return fam


@pytest.mark.parametrize("eta", [0.0, 0.05])
def test_penalized_objective_exact_penalty(eta):
    """Lemma l1_prob_equiv (App. C): with the penalty coefficient 2||C||_inf the penalised
    problem (Eq. prob:l1_ot_primal) over row-stochastic p has the same optimal value as OT
    (eta = 0, part a) and, for eta <= K / log(max_j 1/c_j), as EOT (part b): P^eta(X) is
    >= that value for every row-feasible X and equal to it at the optimal plan (LP plan /
    Sinkhorn plan).  A smaller coefficient lets the greedy plan (every row on its cheapest
    column) fall below the optimum."""
    n, m = 9, 11
    C, r, c = small_points(n, m, seed=17, scale=1.0)
    K = O.sup_norm(C)
    rng = np.random.default_rng(5)
    if eta == 0.0:
        vstar = O.ot_lp(C, r, c)
        Xstar = _lp_plan(C, r, c)
    else:
        assert eta <= K / math.log(1.0 / c.min())
        Xstar, f, g, _ = O.sinkhorn_log(C, r, c, eta, tol=1e-14)
        vstar = O.eot_value(C, Xstar, eta)
    assert abs(O.penalized_objective(Xstar, C, c, K, eta) - vstar) <= 1e-9
    vals = [O.penalized_objective(X, C, c, K, eta) for X in _row_feasible_family(C, r, Xstar, rng)]
    assert min(vals) >= vstar - 1e-10, (min(vals), vstar)
    # without the penalty the greedy plan is below the optimum: the penalty is what lifts it
    assert O.eot_value(C, _row_feasible_family(C, r, Xstar, rng)[0], eta) < vstar


def test_penalty_coefficient_is_exact_where_half_of_it_is_not():
    """The factor 2 of the penalty 2||C||_inf ||col - c||_1 (Eq. prob:l1_ot_primal).  The proof
    of Lemma l1_prob_equiv (b) makes the penalised and the EOT problem share their minimiser
    whenever the penalty coefficient mu is at least ||psi*||_inf for an optimal column
    multiplier psi* (Lemma affine_minimizer); psi* is fixed up to a constant (sum col = sum c),
    so the smallest such norm is half the range of Sinkhorn's column potentials g.  On a
    problem with a tiny c_j and eta = 0.2 K that range lies between 2K and 4K: mu = 2K is
    exact (P^eta >= EOT* on every row-feasible X, = at the optimum), while mu = K is not:
    moving mass delta within a row from the column of max g to the column of min g changes
    the entropic cost by delta (min g - max g) and the penalty by 2 mu delta, a net decrease."""
    w = W.points_problem("t", 8, 9, 2, 17, dist="uniform", marg="random", cost_scale=1.0)
    C = O.cost_matrix(w)
    C = C / C.max()
    K = O.sup_norm(C)
    r = w.r
    c = w.c.copy()
    c[0] = 1e-7
    c /= c.sum()
    eta = 0.2 * K
    Xs, f, g, _ = O.sinkhorn_log(C, r, c, eta, tol=1e-14)
    spread = g.max() - g.min()
    assert 2.2 * K < spread < 3.8 * K, spread
    vstar = O.eot_value(C, Xs, eta)
    assert abs(O.penalized_objective(Xs, C, c, K, eta) - vstar) <= 1e-12
    jhi, jlo = int(g.argmax()), int(g.argmin())
    fam = []
    for i in range(C.shape[0]):
        for frac in (1e-3, 1e-2, 1e-1):
            X = Xs.copy()
            dlt = frac * X[i, jlo]  # small against the receiving entry (c_jlo is tiny)
            X[i, jhi] -= dlt
            X[i, jlo] += dlt
            fam.append(X)
    fam += _row_feasible_family(C, r, Xs, np.random.default_rng(8))
    vals = np.array([O.penalized_objective(X, C, c, K, eta) for X in fam])
    assert vals.min() >= vstar - 1e-12, vals.min() - vstar
    # the same moves with half the coefficient go below the optimum
    half = [O.eot_value(C, X, eta) + K * np.abs(X.sum(0) - c).sum() for X in fam[:2]]
    assert max(half) < vstar


def test_objective_report_uses_the_pinned_penalty():
    """objective_report's P^eta and L are the pinned functions of X^t."""
    C, r, c = small_points(7, 8, seed=3)
    K = O.sup_norm(C)
    st = O.lamp_run(C, r, c, O.LampParams(eta=0.02), 40)
    rep = O.objective_report(C, r, c, K, 0.02, st)
    X = rep["X"]
    assert rep["P_eta"] == O.penalized_objective(X, C, c, K, 0.02)
    assert rep["L"] == O.eot_value(C, X, 0.02)


def test_certificate_terms_of_the_proof():
    """Prop. infeas_bound (a) is the sum of two bounds from its proof (Lemma last_iterate,
    App. D), each checked on its own along a trajectory at every t >= 1:
      Round term  <C, Round(X^t)> - <C, X^t> <= K ||Round(X^t) - X^t||_1 <= 2K res_t
                  (Hoelder, Lemma jason_rounding);
      LAMP term   <C, X^t> - OT* <= -2K <nu^t, col(X^t) - c> + 2K log m / t
                  <= 2K res_t + 2K log m / t.
    certificate_rhs adds the right sides: 4K res_t + 2K log m / t.  The inequality pins the
    constant from below only (a larger constant would still bound the gap)."""
    n, m = 10, 12
    C, r, c = small_points(n, m, seed=29, scale=1.3)
    K = O.sup_norm(C)
    ot = O.ot_lp(C, r, c)
    seen = []

    def rec(s, info):
        if s.t == 0:
            return
        X = r[:, None] * O.dual_to_primal(C, K, s.kappa, s.nu)[0]
        col = X.sum(0)
        res = float(np.abs(col - c).sum())
        Xr = O.round_plan(X, r, c)
        cx, crx = float((C * X).sum()), float((C * Xr).sum())
        assert crx - cx <= K * np.abs(Xr - X).sum() + 1e-12
        assert np.abs(Xr - X).sum() <= 2 * res + 1e-12
        lamp_term = -2 * K * float(s.nu @ (col - c)) + 2 * K * math.log(m) / s.t
        assert cx - ot <= lamp_term + 1e-12
        assert lamp_term <= 2 * K * res + 2 * K * math.log(m) / s.t + 1e-12
        seen.append((crx - ot, O.certificate_rhs(K, res, m, s.t), 2 * K * res + lamp_term))
        assert crx - ot <= 2 * K * res + lamp_term + 1e-12 <= O.certificate_rhs(K, res, m, s.t) + 2e-12

    O.lamp_run(C, r, c, O.LampParams(), 1500, record=rec)
    assert len(seen) == 1499
