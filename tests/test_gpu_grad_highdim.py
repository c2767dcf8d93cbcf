"""lamp_grad for d > 8: the float32 dot form (chunks of 8 coordinates per recompute sweep)
and the tensor-core pass (S = x.y^T and P.Y on tcgen05, one pass per side), against the
oracle's envelope gradient on the same state, and the autograd form (lamp_ot_loss) with
tensor cores against FP64 Sinkhorn on the bf16-rounded points."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_util import GRAD_TOL, dev, gpu_solver, oracle_cost

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,prec,eta", [(16, "fp32", 0.0), (20, "fp32", 0.5), (64, "bf16_tc", 0.0), (33, "bf16_tc", 1.0)])
def test_gradient_high_dim_on_oracle_state(d, prec, eta):
    w = W.points_problem(f"g{d}", 300, 257, d, seed=d, dist="gauss_shift", marg="random", cost_scale=0.05, eta=eta)
    if prec == "bf16_tc":
        w = dataclasses.replace(w, x=W.bf16_round(w.x), y=W.bf16_round(w.y))
    C, s, K = oracle_cost(w)
    st = O.lamp_run(C, w.r, w.c, O.LampParams(eta=eta, K=K), 25)
    sol, _, _ = gpu_solver(w, K=K, scale=s, eta=eta, prec=prec, check_every=5)
    sol.set_state(st.nu, st.theta, st.kappa, st.t)
    dx, dy = sol.grad()
    dx = dx.cpu().numpy().astype(np.float64)
    dy = dy.cpu().numpy().astype(np.float64)
    X = w.r[:, None] * O.dual_to_primal(C, K, st.kappa, st.nu)[0]
    gx, gy = O.grad_envelope(w.x, w.y, X, scale=s)
    assert np.abs(dx - gx).max() <= GRAD_TOL * np.abs(gx).max(), np.abs(dx - gx).max() / np.abs(gx).max()
    assert np.abs(dy - gy).max() <= GRAD_TOL * np.abs(gy).max(), np.abs(dy - gy).max() / np.abs(gy).max()
    # translation invariance of the cost: sum_i dL/dx_i + sum_j dL/dy_j = 0
    tot = np.abs(dx).sum() + np.abs(dy).sum()
    assert np.abs(dx.sum(0) + dy.sum(0)).max() <= 1e-5 * tot
    sol.close()


def test_autograd_form_with_tensor_cores_high_dim():
    import torch
    import paper_2511_11359_gb300 as L

    eta = 1.0
    w = W.points_problem("agtc", 200, 180, 64, seed=9, dist="gauss_shift", marg="uniform", cost_scale=0.05, eta=eta)
    xr, yr = W.bf16_round(w.x), W.bf16_round(w.y)
    x = dev(w.x).requires_grad_(True)
    y = dev(w.y).requires_grad_(True)
    loss = L.lamp_ot_loss(x, y, eta=eta, cost_scale=0.05, prec="bf16_tc", tol=5e-7, max_iter=400000)
    loss.backward()
    C = O.sqeuclid_cost(xr, yr, scale=0.05)
    X, *_ = O.sinkhorn_log(C, w.r, w.c, eta, tol=1e-14)
    gx, gy = O.grad_envelope(xr, yr, X, scale=0.05)
    ref = O.eot_value(C, X, eta)
    assert abs(loss.item() - ref) <= 1e-6 * abs(ref), abs(loss.item() - ref) / abs(ref)
    assert np.abs(x.grad.cpu().numpy() - gx).max() <= GRAD_TOL * np.abs(gx).max()
    assert np.abs(y.grad.cpu().numpy() - gy).max() <= GRAD_TOL * np.abs(gy).max()


@pytest.mark.parametrize("n,m,d,T", [(4096, 3000, 64, 40), (1500, 2200, 17, 300)])
def test_tc_gradient_many_tiles(n, m, d, T):
    """The tensor-core gradient pass with many streamed tiles per CTA, several inner splits
    and ragged tails on both sides (and coordinates zero-padded to 64 for d = 17): dx and dy
    against the oracle's envelope gradient sum_j X_ij dC_ij/dx_i on the oracle's state."""
    w = W.points_problem(f"tcg{n}", n, m, d, seed=n % 97, dist="gauss_shift", marg="random", cost_scale=1.0)
    w = dataclasses.replace(w, x=W.bf16_round(w.x), y=W.bf16_round(w.y))
    C, s, K = oracle_cost(w)
    st = O.lamp_run(C, w.r, w.c, O.LampParams(K=K), T)
    sol, _, _ = gpu_solver(w, K=K, scale=s, prec="bf16_tc", check_every=5)
    sol.set_state(st.nu, st.theta, st.kappa, st.t)
    dx, dy = sol.grad()
    dx = dx.cpu().numpy().astype(np.float64)
    dy = dy.cpu().numpy().astype(np.float64)
    X = w.r[:, None] * O.dual_to_primal(C, K, st.kappa, st.nu)[0]
    gx, gy = O.grad_envelope(w.x, w.y, X, scale=s)
    ex = np.abs(dx - gx).max() / np.abs(gx).max()
    ey = np.abs(dy - gy).max() / np.abs(gy).max()
    print(f"\ntc gradient n={n} m={m} d={d}: rel err dx {ex:.3e} dy {ey:.3e}")
    assert ex <= GRAD_TOL and ey <= GRAD_TOL
    # a second call on the same state gives the same result (no stale partials)
    dx2, dy2 = sol.grad()
    assert np.array_equal(dx2.cpu().numpy(), dx.astype(np.float32))
    sol.close()
