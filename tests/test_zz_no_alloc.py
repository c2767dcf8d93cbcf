"""lamp_marginals_noalloc, the entry point for callers that may not allocate device
memory, against the regular context path (lamp_set_state + lamp_objective +
lamp_get_state) on the same state, through the C ABI, on two calls in a row, and
against the FP64 oracle's marginals of the same (nu, kappa).

Collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_util import LOGZ_TOL, OBJ_TOL, RES_FLOOR, assert_logZ_close, dev, gpu_solver, oracle_cost

pytestmark = pytest.mark.gpu


def _fn():
    import paper_2511_11359_gb300 as L

    f = L._get_lib().lamp_marginals_noalloc
    f.argtypes = [ctypes.POINTER(L._Problem), ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L, f


def _problem(L, w, tensors, scale):
    pr = L._Problem()
    pr.n, pr.m = w.n, w.m
    if w.kind == "dense":
        pr.kind, pr.C, pr.ldc, pr.d = L.COST_DENSE, tensors["C"].data_ptr(), w.m, 0
    else:
        pr.kind, pr.x, pr.y, pr.d = L.COST_SQEUCLID, tensors["x"].data_ptr(), tensors["y"].data_ptr(), w.d
    pr.r, pr.c, pr.cost_scale = tensors["r"].data_ptr(), tensors["c"].data_ptr(), scale
    return pr


@pytest.mark.parametrize("kind", ["sqeuclid", "dense"])
def test_noalloc_matches_context_path_on_two_calls(kind):
    import torch

    L, f = _fn()
    if kind == "sqeuclid":
        w = W.points_problem("na", 300, 257, 3, seed=17, cost_scale=0.5)
    else:
        w = W.dense_problem("na", 290, 1100, seed=18)
    C, scale, K = oracle_cost(w)
    t = {"r": dev(w.r), "c": dev(w.c)}
    if kind == "dense":
        t["C"] = dev(w.C)
    else:
        t["x"], t["y"] = dev(w.x), dev(w.y)
    pr = _problem(L, w, t, scale)
    s, _, _ = gpu_solver(w, check_every=5)
    stream = torch.cuda.current_stream()
    for T in (40, 75):  # two calls in a row, on two different states
        s.iterate(T - (0 if T == 40 else 40))
        obj = s.objective()
        st = s.get_state()
        nu = dev(st["nu"])
        logZ = torch.empty(w.n, dtype=torch.float64, device="cuda")
        col = torch.empty(w.m, dtype=torch.float64, device="cuda")
        cost = torch.empty(1, dtype=torch.float64, device="cuda")
        code = f(ctypes.byref(pr), K, st["kappa"], nu.data_ptr(), logZ.data_ptr(), col.data_ptr(), cost.data_ptr(),
                 ctypes.c_void_p(stream.cuda_stream))
        assert code == L.LAMP_OK, L._get_lib().lamp_last_error(None)
        torch.cuda.synchronize()
        lz = logZ.cpu().numpy()
        cl = col.cpu().numpy()
        assert_logZ_close(lz, st["logZ"], LOGZ_TOL, what=f"noalloc log Z, T={T}")
        assert abs(cost.item() - obj["cost"]) <= OBJ_TOL * abs(obj["cost"])
        assert abs(np.abs(cl - w.c).sum() - obj["col_res"]) <= 1e-6 * obj["col_res"] + RES_FLOOR
        assert abs(cl.sum() - 1.0) <= 1e-6
        # the FP64 oracle on the same (nu, kappa): col(X) and log Z of X = diag(r) p^{1/kappa}(nu)
        ocol, olz = O.marginals_from_state(C, w.r, K, st["kappa"], st["nu"])
        assert_logZ_close(lz, olz, LOGZ_TOL, what=f"noalloc log Z vs oracle, T={T}")
        assert np.abs(cl - ocol).sum() <= 1e-6  # col(X) sums to 1: 1e-6 relative in the L1 norm
        ocost = float((C * (w.r[:, None] * O.dual_to_primal(C, K, st["kappa"], st["nu"])[0])).sum())
        assert abs(cost.item() - ocost) <= OBJ_TOL * abs(ocost)
    s.close()


def test_noalloc_rejects_what_does_not_fit():
    import torch

    L, f = _fn()
    n = m = 1 << 17  # needs far more than the 16 MiB static workspace
    pr = L._Problem()
    pr.n, pr.m, pr.d, pr.kind = n, m, 3, L.COST_SQEUCLID
    pr.x = pr.y = pr.r = pr.c = 0x1000  # never dereferenced: the size check comes first
    pr.cost_scale = 1.0
    code = f(ctypes.byref(pr), 1.0, 1.0, 0x2000, 0x3000, 0x4000, None, None)
    assert code == L.LAMP_E_INVALID
    assert b"scratch" in L._get_lib().lamp_last_error(None)
    pr.d = 16
    assert f(ctypes.byref(pr), 1.0, 1.0, 0x2000, 0x3000, 0x4000, None, None) == L.LAMP_E_UNSUPPORTED
