"""Pin of the oracle's Dt_summand (one summand of D_t, Eq. def:sum_condition) against an
independent re-expression of both of its differences.

* KL part.  For Gibbs-form couplings X = diag(r) p^{eta}(nu), log X_ij = log r_i -
  kappa (C_ij + 2K nu_j) - log Z_i (Eq. def:dual_to_primal), so for any Y with row(Y) = r
      KL(Y || X^{t+1}) - KL(Y || X^t) = (kappa_{t+1} - kappa_t) <Y, C>
          + 2K <col(Y), kappa_{t+1} nu^{t+1} - kappa_t nu^t> + <r, log Z^{t+1} - log Z^t>
  (the masses of X^t and X^{t+1} are both sum r).  The test evaluates this with its own
  log-sum-exp normalisers and Y = Xbar^{t+1} built from them, never forming log X.
* D_Ha part.  D_Ha is the Bregman divergence of h(theta) = sum_j c^alpha_j [(1 + theta_j)/2
  log(1 + theta_j) + (1 - theta_j)/2 log(1 - theta_j)] (Eq. def:DHa_explicit), whose gradient
  is c^alpha atanh(theta): D(u || v) = h(u) - h(v) - <grad h(v), u - v>.

A swapped KL or D_Ha argument, a sign error, or the wrong iterate in any of the four terms
changes the value by far more than the tolerance (checked on the wrong variants below)."""
import numpy as np
import pytest
from scipy.special import logsumexp

import oracle as O


def _h(theta, calpha):
    return float(calpha @ ((1 + theta) / 2 * np.log1p(theta) + (1 - theta) / 2 * np.log1p(-theta)))


def _bregman(u, v, calpha):
    return _h(u, calpha) - _h(v, calpha) - float((calpha * np.arctanh(v)) @ (u - v))


def _lse_rows(C, K, kappa, nu):
    return logsumexp(-kappa * (C + 2.0 * K * nu[None, :]), axis=1)


def _independent(C, r, K, calpha, prev, info, new):
    lz_t = _lse_rows(C, K, prev.kappa, prev.nu)
    lz_1 = _lse_rows(C, K, new.kappa, new.nu)
    lz_b = _lse_rows(C, K, info.kappa_next, info.nubar)
    Xbar = r[:, None] * np.exp(-info.kappa_next * (C + 2.0 * K * info.nubar[None, :]) - lz_b[:, None])
    dkl = ((new.kappa - prev.kappa) * float((Xbar * C).sum())
           + 2.0 * K * float(Xbar.sum(axis=0) @ (new.kappa * new.nu - prev.kappa * prev.nu))
           + float(r @ (lz_1 - lz_t)))
    ddh = _bregman(info.thetabar, info.thetahat, calpha) - _bregman(info.thetabar, prev.theta, calpha)
    return ddh + dkl, Xbar


CASES = [(5, 4, 0.0, 1), (7, 9, 0.0, 2), (6, 6, 0.05, 3), (11, 8, 0.2, 4)]


@pytest.mark.parametrize("n,m,eta,seed", CASES)
def test_dt_summand_matches_independent_form(n, m, eta, seed):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0.0, 1.0, size=(n, m))
    r = rng.uniform(0.2, 1.0, size=n)
    r /= r.sum()
    c = rng.uniform(0.2, 1.0, size=m)
    c /= c.sum()
    P = O.LampParams(eta=eta)
    K, tau1, tau2 = O.resolve_params(C, P)
    calpha = O.calpha_of(c, P.alpha)
    st = O.lamp_initial_state(m)
    checked = 0
    for t in range(40):
        prev = st
        st, info = O.lamp_step(C, r, c, K, tau1, tau2, eta, calpha, P.beta, prev)
        if t == 0:
            continue  # kappa_0 = 0: X^0 is the uniform plan, still covered from t = 1 on
        got = O.Dt_summand(C, r, K, calpha, prev, info, st)
        ref, Xbar = _independent(C, r, K, calpha, prev, info, st)
        scale = 1e-12 + abs(ref)
        assert abs(got - ref) <= 1e-9 * max(scale, 1e-6), (t, got, ref)
        # the pin separates the plausible wrong variants of the summand
        Xs = r[:, None] * O.dual_to_primal(C, K, prev.kappa, prev.nu)[0]
        Xn = r[:, None] * O.dual_to_primal(C, K, st.kappa, st.nu)[0]
        wrong = [
            O.D_Ha(info.thetabar, info.thetahat, calpha) - O.D_Ha(info.thetabar, prev.theta, calpha)
            + O.KL(Xn, Xbar) - O.KL(Xs, Xbar),                                  # KL arguments swapped
            O.D_Ha(info.thetahat, info.thetabar, calpha) - O.D_Ha(prev.theta, info.thetabar, calpha)
            + O.KL(Xbar, Xn) - O.KL(Xbar, Xs),                                  # D_Ha arguments swapped
            O.D_Ha(info.thetabar, info.thetahat, calpha) - O.D_Ha(info.thetabar, prev.theta, calpha)
            - O.KL(Xbar, Xn) + O.KL(Xbar, Xs),                                  # KL sign
            O.D_Ha(info.thetabar, st.theta, calpha) - O.D_Ha(info.thetabar, prev.theta, calpha)
            + O.KL(Xbar, Xn) - O.KL(Xbar, Xs),                                  # clipped theta^{t+1} for thetahat
        ]
        for k, wv in enumerate(wrong):
            if k == 3 and np.array_equal(st.theta, info.thetahat):
                continue  # no clipping at this step: the variant coincides
            assert abs(wv - ref) > 1e3 * 1e-9 * max(scale, 1e-6), (t, k)
        checked += 1
    assert checked == 39


def test_kl_difference_identity_on_arbitrary_row_feasible_plan():
    """The KL identity used above holds for any Y with row(Y) = r, not only Xbar: checked on
    a random row-feasible plan against the oracle's elementwise KL."""
    rng = np.random.default_rng(8)
    n, m = 6, 5
    C = rng.uniform(0.0, 1.0, size=(n, m))
    r = np.full(n, 1.0 / n)
    c = np.full(m, 1.0 / m)
    P = O.LampParams()
    K, tau1, tau2 = O.resolve_params(C, P)
    st = O.lamp_run(C, r, c, P, 7)
    nxt = O.lamp_run(C, r, c, P, 1, state=st)
    Y = rng.uniform(0.1, 1.0, size=(n, m))
    Y *= (r / Y.sum(axis=1))[:, None]
    X0 = r[:, None] * O.dual_to_primal(C, K, st.kappa, st.nu)[0]
    X1 = r[:, None] * O.dual_to_primal(C, K, nxt.kappa, nxt.nu)[0]
    lhs = O.KL(Y, X1) - O.KL(Y, X0)
    rhs = ((nxt.kappa - st.kappa) * float((Y * C).sum())
           + 2.0 * K * float(Y.sum(axis=0) @ (nxt.kappa * nxt.nu - st.kappa * st.nu))
           + float(r @ (_lse_rows(C, K, nxt.kappa, nxt.nu) - _lse_rows(C, K, st.kappa, st.nu))))
    assert abs(lhs - rhs) <= 1e-11 * (1.0 + abs(rhs))
