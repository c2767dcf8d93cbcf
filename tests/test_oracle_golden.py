"""The oracle's exact solvers and LAMP's certified bracket against the closed-form values of
tests/golden/closed_form_ot.json (derived by hand from the problem definitions; the paper
prints no worked numerical example)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "closed_form_ot.json")
with open(GOLDEN) as f:
    FIX = json.load(f)


def _problem(case):
    if "C" in case:
        return np.asarray(case["C"], float), np.asarray(case["r"], float), np.asarray(case["c"], float)
    x, y = np.asarray(case["x"], float), np.asarray(case["y"], float)
    d = np.abs(x[:, None] - y[None, :])
    C = d if case["cost"] == "abs" else d ** 2
    n = len(x)
    return C, np.full(n, 1.0 / n), np.full(len(y), 1.0 / len(y))


@pytest.mark.parametrize("case", FIX["cases"], ids=[c["name"] for c in FIX["cases"]])
def test_lp_value_equals_closed_form(case):
    C, r, c = _problem(case)
    assert O.ot_lp(C, r, c) == pytest.approx(case["ot"], abs=1e-12)


@pytest.mark.parametrize("case", FIX["cases"], ids=[c["name"] for c in FIX["cases"]])
def test_lamp_certificate_brackets_closed_form(case):
    """eta = 0: Round(X^T) is feasible, so <C, Round(X^T)> >= OT, and Prop. infeas_bound (a)
    bounds the excess by the certificate 4K ||col - c||_1 + 2K log m / T."""
    C, r, c = _problem(case)
    P = O.LampParams()
    K = O.sup_norm(C)
    for T in (50, 400):
        st = O.lamp_run(C, r, c, P, T)
        X = r[:, None] * O.dual_to_primal(C, K, st.kappa, st.nu)[0]
        Xr = O.round_plan(X, r, c)
        cost = float((C * Xr).sum())
        cert = O.certificate_rhs(K, float(np.abs(X.sum(axis=0) - c).sum()), C.shape[1], T)
        assert cost >= case["ot"] - 1e-12
        assert cost - case["ot"] <= cert + 1e-12


@pytest.mark.parametrize("case", FIX["entropic"], ids=[c["name"] for c in FIX["entropic"]])
def test_sinkhorn_plan_and_value_equal_closed_form(case):
    C, r, c = (np.asarray(case[k], float) for k in ("C", "r", "c"))
    eta = case["eta"]
    e = math.exp(1.0 / eta)
    a = e / (2.0 * (1.0 + e))
    Xcf = np.array([[a, 0.5 - a], [0.5 - a, a]])
    X, *_ = O.sinkhorn_log(C, r, c, eta, tol=1e-14)
    assert np.abs(X - Xcf).max() <= 1e-12
    H = -float((Xcf * np.log(Xcf)).sum())
    assert O.eot_value(C, X, eta) == pytest.approx(float((C * Xcf).sum()) - eta * H, abs=1e-12)
