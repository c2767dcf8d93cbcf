"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins catch them.

Each mutation rewrites one line of one oracle function (a dropped factor, a wrong
sign or index, a transposed operand), installs the mutated function in the oracle
module for the duration of the test, and runs the pin that is meant to catch it:
the pin must fail."""
import inspect
import math
import textwrap

import numpy as np
import pytest

import oracle.lamp_oracle as OL
import tests.test_oracle_dt as DT
import tests.test_oracle_golden as GOLD
import tests.test_oracle_pins as PINS


def _mutate(monkeypatch, fname, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(OL, fname)))
    assert old in src, (fname, old)
    ns = {}
    exec(compile(src.replace(old, new, 1), f"<mutant {fname}>", "exec"), OL.__dict__, ns)
    monkeypatch.setattr(OL, fname, ns[fname])
    # the tests import the package namespace; keep it in sync
    import oracle
    monkeypatch.setattr(oracle, fname, ns[fname], raising=False)


MUTANTS = [
    # (function, original text, mutated text, pin that must fail, pin args)
    ("dual_mirror_map", "2.0 * tau * K", "tau * K", PINS.test_dual_mirror_map_is_the_argmax, ()),
    ("dual_mirror_map", "(colr - c)", "(c - colr)", PINS.test_dual_mirror_map_is_the_argmax, ()),
    ("dual_to_primal", "2.0 * K * nu", "K * nu", PINS.test_lamp_equals_explicit_pdmp, (16, 16, 2, 0.0)),
    ("log_normalizers", "return mx + np.log(", "return np.log(", PINS.test_lamp_equals_explicit_pdmp, (16, 16, 2, 0.0)),
    ("kappa_next", "tau1 + kappa * (1.0 - tau1 * eta)", "tau1 + kappa * (1.0 + tau1 * eta)",
     PINS.test_kappa_recursion_matches_closed_form, (0.05,)),
    ("lamp_step", "nubar = nu + w * (theta - nu)", "nubar = nu + w * (theta + nu)",
     PINS.test_lamp_equals_explicit_pdmp, (16, 16, 2, 0.0)),
    ("lamp_step", "thetahat = dual_mirror_map(theta, B,", "thetahat = dual_mirror_map(thetabar, B,",
     PINS.test_lamp_equals_explicit_pdmp, (16, 16, 2, 0.0)),
    ("lamp_step", "w = tau1 / kap1", "w = tau1 / (kap1 + tau1)",
     PINS.test_lamp_equals_explicit_pdmp, (7, 5, 1, 1e-2)),
    ("lamp_step", "XA = r[:, None] * pA", "XA = pA / pA.shape[0]", PINS.test_uniform_start, (5, 9)),
    ("col_r", "(r[:, None] * p).sum(axis=0)", "(r[:, None] * p).sum(axis=1)",
     PINS.test_lamp_equals_explicit_pdmp, (16, 16, 2, 0.0)),
    ("tclip", "np.tanh(beta / 2.0)", "np.tanh(beta)", PINS.test_tclip_bounds, ()),
    ("round_factors", "X2 = X1 * y[None, :]", "X2 = X1", PINS.test_round_is_feasible_and_within_bound, (0,)),
    ("l1_cost", "out += np.abs(", "out += (", PINS.test_point_costs_match_scipy_distances, ()),
    ("linf_cost", "np.maximum(out, np.abs(", "np.maximum(out, (", PINS.test_point_costs_match_scipy_distances, ()),
    ("cosine_cost", "(nx[:, None] * ny[None, :])", "(nx[:, None] * nx[:, None])", PINS.test_point_costs_match_scipy_distances, ()),
    ("round_plan", "np.outer(dr, dc) / l1", "np.outer(dc, dr).T / l1 * 0.5", PINS.test_round_is_feasible_and_within_bound, (0,)),
    ("entropy_from_normalizers", "2.0 * K * kappa", "K * kappa", PINS.test_entropy_identity, (0.0,)),
    ("saddle_dual", "- 2.0 * K * (c @ theta)", "+ 2.0 * K * (c @ theta)",
     PINS.test_saddle_dual_strong_duality_at_lp_potentials, ()),
    ("saddle_dual", "const = -eta * (", "const = 0.0 * (",
     PINS.test_entropic_saddle_dual_equals_eot_value_at_lamp_limit, ()),
    ("saddle_dual", "rowpart = Z.min(axis=1)", "rowpart = Z.mean(axis=1)",
     PINS.test_saddle_dual_strong_duality_at_lp_potentials, ()),
    ("sinkhorn_log", "eta * (lc -", "eta * (lr.mean() + lc -", PINS.test_sinkhorn_pinned_to_lp, ()),
    ("certificate_rhs", "2.0 * K * np.log(m) / t", "2.0 * K * np.log(m) / t ** 2",
     PINS.test_certificate_log_term_is_one_over_t, ()),
    ("grad_envelope", "rowX[:, None] * x - X @ y", "rowX[:, None] * x - X.T[: x.shape[0], : y.shape[0]] @ y[: X.shape[0]]",
     PINS.test_envelope_gradient_matches_fd_of_sinkhorn_value, ()),
    ("Dt_summand", "+ KL(Xbar, Xnew) - KL(Xbar, Xs)", "+ KL(Xnew, Xbar) - KL(Xbar, Xs)",
     DT.test_dt_summand_matches_independent_form, (7, 9, 0.0, 2)),
    ("Dt_summand", "dual_to_primal(C, K, new.kappa, new.nu)", "dual_to_primal(C, K, new.kappa, prev.nu)",
     DT.test_dt_summand_matches_independent_form, (6, 6, 0.05, 3)),
    ("Dt_summand", "- D_Ha(info.thetabar, prev.theta, calpha)", "+ D_Ha(info.thetabar, prev.theta, calpha)",
     DT.test_dt_summand_matches_independent_form, (5, 4, 0.0, 1)),
    ("penalized_objective", "2.0 * K * np.abs", "K * np.abs",
     PINS.test_penalty_coefficient_is_exact_where_half_of_it_is_not, ()),
    ("penalized_objective", "2.0 * K * np.abs", "0.0 * K * np.abs", PINS.test_penalized_objective_exact_penalty, (0.0,)),
    ("penalized_objective", "- eta * entropy(X)", "+ eta * entropy(X)", PINS.test_penalized_objective_exact_penalty,
     (0.05,)),
    ("penalized_objective", "X.sum(axis=0) - c", "X.sum(axis=1)[: c.shape[0]] - c",
     PINS.test_penalized_objective_exact_penalty, (0.0,)),
    ("objective_report", '"P_eta": penalized_objective(X, C, c, K, eta)', '"P_eta": cost + K * col_res - eta * H',
     PINS.test_objective_report_uses_the_pinned_penalty, ()),
    ("eot_value", "- eta * entropy(X)", "+ eta * entropy(X)",
     GOLD.test_sinkhorn_plan_and_value_equal_closed_form, (GOLD.FIX["entropic"][0],)),
    ("entropy", "np.log(Xp)", "np.log2(Xp)",
     GOLD.test_sinkhorn_plan_and_value_equal_closed_form, (GOLD.FIX["entropic"][0],)),
]


@pytest.mark.parametrize("fname,old,new,pin,args", MUTANTS, ids=[f"{m[0]}:{i}" for i, m in enumerate(MUTANTS)])
def test_pin_catches_mutant(monkeypatch, fname, old, new, pin, args):
    _mutate(monkeypatch, fname, old, new)
    with pytest.raises((AssertionError, ValueError, FloatingPointError, IndexError)):
        with np.errstate(all="ignore"):
            pin(*args)


def test_unmutated_pins_pass():
    # the same pin invocations pass on the real oracle
    for _, _, _, pin, args in MUTANTS:
        pin(*args)
