"""Failure detection on the GPU without a fault: the bounded mbarrier wait of the
tensor-core sweeps, run on a barrier that nothing arrives on, gives up after its poll
limit, records LAMP_E_TIMEOUT in the device status word and returns; the device stays
usable (a solve right after it converges)."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import gpu_solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("polls", [1, 1000, 1 << 16])
def test_bounded_wait_gives_up_and_reports_timeout(polls):
    import paper_2511_11359_gb300 as L

    assert L.selftest_wait_timeout(polls) == L.LAMP_E_TIMEOUT


def test_device_usable_after_a_timed_out_wait():
    import paper_2511_11359_gb300 as L

    assert L.selftest_wait_timeout(64) == L.LAMP_E_TIMEOUT
    w = W.points_problem("after_timeout", 200, 180, 64, seed=3, dist="gauss_shift", marg="uniform")
    for prec in ("bf16_tc", "fp32"):
        s, _, _ = gpu_solver(w, prec=prec, tol=1e-5, max_iter=20000, check_every=50)
        res = s.solve()
        assert res["converged"] and res["infeas"] <= 1e-5 and res["status"] == 0
        s.close()
