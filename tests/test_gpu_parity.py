"""GPU path vs the FP64 oracle on identical seeded inputs (all through the C ABI)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_util import (GRAD_TOL, LOGZ_TOL, OBJ_TOL, POT_TOL, RES_FLOOR, assert_logZ_close, assert_pot_close,
                            cost_slack, dev, gpu_solver, oracle_cost)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2511_11359_gb300 as L  # noqa: F401


POINT_CASES = [
    # (name, n, m, d, dist, marg, scale, eta)
    ("plain2d", 256, 256, 2, "uniform", "random", -1.0, 0.0),
    ("ragged3d", 300, 131, 3, "uniform", "random", 1.0, 0.0),
    ("sphere_eta", 200, 257, 3, "sphere", "uniform", 1.0, 1e-2),
    ("hd64", 160, 200, 64, "gauss_shift", "uniform", 1.0, 0.0),
    ("hd17", 129, 130, 17, "gauss_shift", "random", 0.05, 0.0),
]


@pytest.mark.parametrize("case", POINT_CASES, ids=[c[0] for c in POINT_CASES])
def test_trajectory_points(case):
    name, n, m, d, dist, marg, scale, eta = case
    w = W.points_problem(name, n, m, d, seed=sum(name.encode()) % 1000, dist=dist, marg=marg, cost_scale=scale, eta=eta)
    s, C, K = gpu_solver(w, eta=eta, check_every=7)
    P = O.LampParams(eta=eta, K=K)
    done = 0
    st_ref = None
    for T in (1, 10, 100):
        s.iterate(T - done)
        st_ref = O.lamp_run(C, w.r, w.c, P, T - done, state=st_ref)
        done = T
        assert_pot_close(s.get_state(), st_ref, what=f"{name} T={T}")
    s.close()


DENSE_CASES = [
    # rows 16-byte multiples apart (m % 4 == 0) take the TMA-fed sweeps (32 x 256 tiles):
    # grid16, dense_rand_eta and dense_tma_ragged (ragged row blocks and column tiles);
    # m = 1029 takes the plain-load sweeps
    ("grid16", "grid", 16, 1e-3),
    ("dense_rand", "rand", (173, 1029), 0.0),
    ("dense_rand_eta", "rand", (64, 2100), 5e-2),
    ("dense_tma_ragged", "rand", (300, 1100), 0.0),
]


def dense_workload(kind, size, eta, seed=7):
    if kind == "grid":
        w = W.image_grid(side=size, seed=seed)
        w.eta = eta
        return w
    return W.dense_problem("d", size[0], size[1], seed, eta=eta)


@pytest.mark.parametrize("case", DENSE_CASES, ids=[c[0] for c in DENSE_CASES])
def test_trajectory_dense(case):
    name, kind, size, eta = case
    w = dense_workload(kind, size, eta)
    s, C, K = gpu_solver(w, eta=eta, check_every=5)
    P = O.LampParams(eta=eta, K=K)
    done, st_ref = 0, None
    for T in (1, 10, 100):
        s.iterate(T - done)
        st_ref = O.lamp_run(C, w.r, w.c, P, T - done, state=st_ref)
        done = T
        assert_pot_close(s.get_state(), st_ref, what=f"{name} T={T}")
    s.close()


@pytest.mark.parametrize("n,m", [(1024, 512), (64, 4096), (1000, 4100)])
def test_dense_split_sweeps(n, m):
    """Stored costs whose TMA-fed sweeps split the inner dimension over several CTAs:
    1024 x 512 (column sweep: 4 row splits), 64 x 4096 (row sweep: 2 column splits),
    1000 x 4100 (both, ragged)."""
    w = W.dense_problem("sp", n, m, seed=n + m)
    s, C, K = gpu_solver(w, check_every=5)
    P = O.LampParams(K=K)
    done, st_ref = 0, None
    for T in (1, 10, 30):
        s.iterate(T - done)
        st_ref = O.lamp_run(C, w.r, w.c, P, T - done, state=st_ref)
        done = T
        assert_pot_close(s.get_state(), st_ref, what=f"dense split {n}x{m} T={T}")
    s.close()


@pytest.mark.parametrize("ldc", [304, 301])
def test_dense_with_leading_dimension(ldc):
    """C as an n x m view of a wider row-major array: ldc = 304 keeps rows 16-byte multiples
    apart (TMA-fed sweeps), ldc = 301 does not (plain-load sweeps); both match the oracle on
    the n x m cost."""
    import torch

    w = W.dense_problem("ld", 257, 300, seed=5)
    wide = np.zeros((w.n, ldc), dtype=np.float32)
    wide[:, : w.m] = w.C
    wide[:, w.m:] = 7.0  # never read
    Cd = torch.from_numpy(wide).cuda()[:, : w.m]
    C, _, K = oracle_cost(w)
    import paper_2511_11359_gb300 as L

    s = L.Lamp(dev(w.r), dev(w.c), C=Cd, K=K, check_every=4)
    T = 30
    s.iterate(T)
    ref = O.lamp_run(C, w.r, w.c, O.LampParams(K=K), T)
    assert_pot_close(s.get_state(), ref, what=f"dense ldc={ldc}")
    s.close()


@pytest.mark.parametrize("n,m", [(1, 1), (1, 7), (7, 1), (2, 3), (37, 1000), (129, 127), (1000, 37)])
@pytest.mark.parametrize("kind", ["sqeuclid", "dense"])
def test_ragged_and_degenerate_sizes(n, m, kind):
    if kind == "dense":
        w = W.dense_problem("rg", n, m, seed=n * 31 + m)
    else:
        w = W.points_problem("rg", n, m, 3, seed=n * 31 + m, cost_scale=1.0)
    C, _, K = oracle_cost(w)
    if K == 0.0:  # n = m = 1 with identical points cannot happen with these seeds
        pytest.skip("zero cost")
    s, C, K = gpu_solver(w, check_every=3)
    T = 20
    s.iterate(T)
    ref = O.lamp_run(C, w.r, w.c, O.LampParams(K=K), T)
    assert_pot_close(s.get_state(), ref, what=f"{kind} {n}x{m}")
    obj = s.objective()
    rep = O.objective_report(C, w.r, w.c, K, 0.0, ref)
    assert abs(obj["cost"] - rep["cost"]) <= OBJ_TOL * abs(rep["cost"]) + 1e-12
    assert abs(obj["col_res"] - rep["col_res"]) <= 1e-6 * rep["col_res"] + RES_FLOOR
    s.close()


@pytest.mark.parametrize("eta", [0.0, 0.02])
def test_objective_and_logZ_match_oracle(eta):
    w = W.plain_2d(n=200, m=170, seed=3)
    s, C, K = gpu_solver(w, eta=eta, check_every=11)
    T = 150
    s.iterate(T)
    obj = s.objective()
    st = s.get_state()
    ref = O.lamp_run(C, w.r, w.c, O.LampParams(eta=eta, K=K), T)
    rep = O.objective_report(C, w.r, w.c, K, eta, ref)
    assert st["t"] == T
    assert_logZ_close(st["logZ"], rep["logZ"], what="logZ")
    assert abs(obj["cost"] - rep["cost"]) <= OBJ_TOL * rep["cost"]
    assert abs(obj["entropy"] - rep["entropy"]) <= 1e-6 * abs(rep["entropy"])
    assert abs(obj["P_eta"] - rep["P_eta"]) <= 1e-6 * abs(rep["P_eta"]) + 1e-9
    assert abs(obj["col_res"] - rep["col_res"]) <= 1e-6 * rep["col_res"] + RES_FLOOR
    assert obj["row_res"] == 0.0 and obj["K"] == K
    if eta == 0.0:
        assert abs(obj["certificate"] - rep["certificate"]) <= 1e-6 * rep["certificate"]
    else:
        assert math.isnan(obj["certificate"])


@pytest.mark.parametrize("T0", [500, 3000])
@pytest.mark.parametrize("kind", ["dense", "sqeuclid_dyadic", "sqeuclid"])
def test_single_step_at_large_kappa(T0, kind):
    """One iteration from an oracle state with kappa = T0/(2K): the compensated
    exponent keeps the float32 sweeps accurate although lambda C = O(T0).
    dense and sqeuclid_dyadic give the kernels the oracle's exact cost (dyadic
    coordinates make every squared distance exact in float32): tolerance 1e-5.
    sqeuclid on random points adds the float32 cost error times kappa."""
    if kind == "dense":
        w = W.dense_problem("lk", 64, 80, seed=5)
    elif kind == "sqeuclid_dyadic":
        w = W.points_problem("lk", 64, 80, 2, seed=5, cost_scale=1.0, grid_step=64)
    else:
        w = W.points_problem("lk", 64, 80, 2, seed=5, cost_scale=-1.0)
    s, C, K = gpu_solver(w, check_every=1)
    P = O.LampParams(K=K)
    st0 = O.lamp_run(C, w.r, w.c, P, T0)
    tol = POT_TOL if kind != "sqeuclid" else cost_slack(w, st0.kappa)
    s.set_state(st0.nu, st0.theta, st0.kappa, st0.t)
    s.iterate(1)
    g = s.get_state()
    K_, tau1, tau2 = O.resolve_params(C, P)
    ref1, info = O.lamp_step(C, w.r, w.c, K_, tau1, tau2, 0.0, O.calpha_of(w.c, 0.01), 1.1, st0)
    assert_pot_close(g, ref1, tol=tol, what=f"step at t={T0}")
    assert g["t"] == T0 + 1 and g["kappa"] == pytest.approx(ref1.kappa, rel=1e-15)
    # log Z of X^{T0}: absolute error small although |log Z| ~ kappa
    s2, _, _ = gpu_solver(w, check_every=1)
    s2.set_state(st0.nu, st0.theta, st0.kappa, st0.t)
    s2.objective()
    lz = s2.get_state()["logZ"]
    assert np.abs(lz - info.logZ_A).max() <= (1e-5 if kind != "sqeuclid" else 1e-5 + 4 * st0.kappa * (tol - POT_TOL))
    s.close()
    s2.close()


@pytest.mark.parametrize("kind", ["plain_2d", "dyadic"])
def test_solve_stops_where_the_oracle_does(kind):
    if kind == "plain_2d":
        w = W.plain_2d(n=128, m=128, seed=9)
    else:
        w = W.points_problem("dy", 128, 128, 2, seed=9, cost_scale=1.0, grid_step=64)
    tol = 1e-6
    s, C, K = gpu_solver(w, tol=tol, max_iter=200000, check_every=64)
    res = s.solve(allow_not_converged=False)
    st_ref, info, conv = O.lamp_solve(C, w.r, w.c, O.LampParams(K=K), tol, 200000)
    assert conv and res["converged"]
    assert res["infeas"] <= tol and res["iters"] >= 1
    assert abs(res["iters"] - st_ref.t) <= max(2, 0.02 * st_ref.t), (res["iters"], st_ref.t)
    # the oracle's own residual at the GPU's final state
    g = s.get_state()
    colX, _ = O.marginals_from_state(C, w.r, K, g["kappa"], g["nu"])
    slack = 0.0 if kind == "dyadic" else 4 * g["kappa"] * (cost_slack(w, 1.0) - POT_TOL)
    assert np.abs(colX - w.c).sum() <= 1.05 * tol + RES_FLOOR + slack
    s.close()


def test_uniform_marginals_do_not_stop_at_the_start():
    """With uniform c the Alg. 2 start X^0 = diag(r)/m is exactly feasible; the
    termination rule starts at t = 1 (oracle and GPU alike)."""
    w = W.points_problem("u", 96, 96, 3, seed=3, dist="gauss_shift", marg="uniform", cost_scale=1.0)
    s, C, K = gpu_solver(w, tol=1e-6, max_iter=100000, check_every=50)
    res = s.solve(allow_not_converged=False)
    st_ref, info, conv = O.lamp_solve(C, w.r, w.c, O.LampParams(K=K), 1e-6, 100000)
    assert res["iters"] >= 1 and st_ref.t >= 1 and conv
    # where the residual curve is flat near tol, float32 and float64 cross it at
    # somewhat different t; what is fixed is that the GPU's state meets the rule
    # under the oracle's arithmetic too (up to the float32 cost error at kappa)
    assert abs(res["iters"] - st_ref.t) <= 0.25 * st_ref.t
    g = s.get_state()
    colX, _ = O.marginals_from_state(C, w.r, K, g["kappa"], g["nu"])
    slack = 4 * g["kappa"] * (cost_slack(w, 1.0) - POT_TOL)
    assert np.abs(colX - w.c).sum() <= 1.05e-6 + RES_FLOOR + slack
    s.close()


def test_not_converged_status_and_result():
    import paper_2511_11359_gb300 as L

    w = W.plain_2d(n=64, m=64, seed=2)
    s, C, K = gpu_solver(w, tol=1e-12, max_iter=37, check_every=10)
    res = s.solve(allow_not_converged=True)
    assert not res["converged"] and res["iters"] == 37 and res["status"] == L.LAMP_E_NOT_CONVERGED
    ref = O.lamp_run(C, w.r, w.c, O.LampParams(K=K), 37)
    assert_pot_close(s.get_state(), ref, what="max_iter")
    with pytest.raises(L.LampError) as e:
        s.solve(allow_not_converged=False)
    assert e.value.code == L.LAMP_E_NOT_CONVERGED
    s.close()


@pytest.mark.parametrize("kind", ["sqeuclid", "dense"])
def test_checkpoint_resume_is_bitwise(kind):
    w = W.plain_2d(n=150, m=140, seed=4) if kind == "sqeuclid" else W.dense_problem("ck", 150, 140, seed=4)
    a, C, K = gpu_solver(w, check_every=4)
    a.iterate(37)
    ck = a.get_state()
    a.iterate(25)
    end_a = a.get_state()
    b, _, _ = gpu_solver(w, check_every=9)
    b.set_state(ck["nu"], ck["theta"], ck["kappa"], ck["t"], ck["row_shifts"])
    b.iterate(25)
    end_b = b.get_state()
    assert end_a["t"] == end_b["t"] == 62
    assert np.array_equal(end_a["nu"], end_b["nu"]) and np.array_equal(end_a["theta"], end_b["theta"])
    # without the shifts the restore is re-primed: equal to the potential tolerance
    c_, _, _ = gpu_solver(w, check_every=9)
    c_.set_state(ck["nu"], ck["theta"], ck["kappa"], ck["t"])
    c_.iterate(25)
    end_c = c_.get_state()
    assert np.abs(end_c["nu"] - end_a["nu"]).max() <= POT_TOL
    for s in (a, b, c_):
        s.close()


@pytest.mark.parametrize("kind", ["sqeuclid", "dense", "sqeuclid_norm"])
def test_K_pass(kind):
    import paper_2511_11359_gb300 as L

    if kind == "dense":
        w = W.dense_problem("k", 300, 517, seed=12)
        s = L.Lamp(dev(w.r), dev(w.c), C=dev(w.C))
        assert s.objective()["K"] == float(w.C.max())
    else:
        w = W.points_problem("k", 333, 250, 5, seed=13, dist="gauss_shift", cost_scale=-1.0 if kind.endswith("norm") else 2.5)
        s = L.Lamp(dev(w.r), dev(w.c), x=dev(w.x), y=dev(w.y), cost_scale=w.cost_scale)
        D = O.sqeuclid_cost(w.x, w.y)
        Kref = 1.0 if w.cost_scale < 0 else 2.5 * D.max()
        assert s.objective()["K"] == pytest.approx(Kref, rel=2e-6)
    s.close()


def test_invalid_inputs_on_gpu():
    import paper_2511_11359_gb300 as L
    import torch

    w = W.plain_2d(n=32, m=40, seed=1)
    x, y = dev(w.x), dev(w.y)
    bad_r = dev(w.r * 1.01)
    with pytest.raises(L.LampError) as e:
        L.Lamp(bad_r, dev(w.c), x=x, y=y)
    assert e.value.code == L.LAMP_E_INVALID
    zr = w.r.copy()
    zr[0] = 0.0
    zr /= zr.sum()
    with pytest.raises(L.LampError):
        L.Lamp(dev(zr), dev(w.c), x=x, y=y)
    Cneg = np.ones((32, 40), np.float32)
    Cneg[3, 4] = -1.0
    with pytest.raises(L.LampError) as e:
        L.Lamp(dev(w.r), dev(w.c), C=dev(Cneg))
    assert e.value.code == L.LAMP_E_INVALID
    Cnan = np.ones((32, 40), np.float32)
    Cnan[0, 0] = np.nan
    with pytest.raises(L.LampError):
        L.Lamp(dev(w.r), dev(w.c), C=dev(Cnan))
    s = L.Lamp(dev(w.r), dev(w.c), x=x, y=y, cost_scale=-1.0)
    with pytest.raises(L.LampError):
        s.set_state(np.full(40, 1.5), np.zeros(40), 1.0, 3)
    with pytest.raises(L.LampError):
        s.iterate(-1)
    s.close()


def test_gradient_matches_oracle_envelope_and_fd():
    """Envelope gradient at the entropic optimum vs the oracle (Sinkhorn plan) and vs
    central finite differences of the FP64 Sinkhorn value."""
    eta = 0.05
    w = W.diffloss(n=150, seed=8)
    s, C, K = gpu_solver(w, eta=eta, tol=5e-7, max_iter=400000, check_every=200)
    res = s.solve(allow_not_converged=False)
    dx, dy = s.grad()
    dx, dy = dx.cpu().numpy().astype(np.float64), dy.cpu().numpy().astype(np.float64)
    X, f, g, _ = O.sinkhorn_log(C, w.r, w.c, eta, tol=1e-14)
    gx, gy = O.grad_envelope(w.x, w.y, X)
    assert np.abs(dx - gx).max() <= GRAD_TOL * np.abs(gx).max()
    assert np.abs(dy - gy).max() <= GRAD_TOL * np.abs(gy).max()
    x64 = w.x.astype(np.float64)
    y64 = w.y.astype(np.float64)
    h = 1e-5
    for (i, k) in [(0, 0), (77, 2), (149, 1)]:
        vals = []
        for sg in (1, -1):
            xp = x64.copy()
            xp[i, k] += sg * h
            Cp = O.sqeuclid_cost(xp, y64)
            Xp, *_ = O.sinkhorn_log(Cp, w.r, w.c, eta, tol=1e-14, f0=f, g0=g)
            vals.append(O.eot_value(Cp, Xp, eta))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(dx[i, k] - fd) <= GRAD_TOL * max(abs(fd), np.abs(gx).max() * 1e-2)
    s.close()


def test_autograd_function():
    import torch
    import paper_2511_11359_gb300 as L

    w = W.diffloss(n=96, seed=21)
    x = dev(w.x).requires_grad_(True)
    y = dev(w.y).requires_grad_(True)
    loss = L.lamp_ot_loss(x, y, eta=0.05, tol=5e-7, max_iter=400000)
    (2.0 * loss).backward()
    C = O.sqeuclid_cost(w.x, w.y)
    X, *_ = O.sinkhorn_log(C, w.r, w.c, 0.05, tol=1e-14)
    gx, gy = O.grad_envelope(w.x, w.y, X)
    assert abs(loss.item() - O.eot_value(C, X, 0.05)) <= 1e-6 * abs(O.eot_value(C, X, 0.05))
    assert np.abs(x.grad.cpu().numpy() - 2 * gx).max() <= GRAD_TOL * 2 * np.abs(gx).max()
    assert np.abs(y.grad.cpu().numpy() - 2 * gy).max() <= GRAD_TOL * 2 * np.abs(gy).max()


def test_host_buffer_entry_point():
    import paper_2511_11359_gb300 as L

    w = W.plain_2d(n=100, m=90, seed=6)
    C, sc, K = oracle_cost(w)
    h = L.LampHost(w.r, w.c, x=w.x, y=w.y, cost_scale=sc, K=K, check_every=5)
    nu = np.empty(90)
    inf = h.step(30, nu_out=nu)
    ref = O.lamp_run(C, w.r, w.c, O.LampParams(K=K), 30)
    assert np.abs(nu - ref.nu).max() <= POT_TOL
    rec = []
    O.lamp_run(C, w.r, w.c, O.LampParams(K=K), 30, record=lambda st, i: rec.append(i.res))
    assert inf == pytest.approx(rec[-1], rel=1e-5)
    h.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16_tc"])
def test_host_buffer_steps_repeat_the_device_context(prec):
    """lamp_step_host re-uploads the host inputs (and re-converts them to bf16 for the
    tensor-core path) before each step: three steps of 4 iterations give bit for bit the
    state of a context on device inputs after 12 iterations."""
    import torch
    import paper_2511_11359_gb300 as L

    w = W.highdim(n=700, m=650, d=16, seed=9)
    h = L.LampHost(w.r, w.c, x=w.x, y=w.y, prec=prec, check_every=4)
    nu = np.empty(650)
    for _ in range(3):
        inf = h.step(4, nu_out=nu)
    h.close()
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    s = L.Lamp(t(w.r), t(w.c), x=t(w.x), y=t(w.y), prec=prec, check_every=4)
    s.iterate(12)
    st = s.get_state()
    s.close()
    assert np.array_equal(nu, st["nu"])
    assert math.isfinite(inf) and inf > 0.0
