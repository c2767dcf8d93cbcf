"""The seeded input generators produce the five workloads' stated shapes and distributions
(sizes, cost normalisation, point distributions, marginals, eta, tolerance), identically for
a given seed."""
import numpy as np
import pytest

import workloads as W


def _marginal_ok(v, n):
    assert v.shape == (n,) and v.dtype == np.float64
    assert np.all(v > 0) and abs(v.sum() - 1.0) <= 1e-12


def test_plain_2d():
    w = W.plain_2d()
    assert (w.n, w.m, w.d, w.eta, w.tol) == (256, 256, 2, 0.0, 1e-6)
    assert w.x.dtype == np.float32 and w.x.min() >= 0 and w.x.max() <= 1 and w.y.max() <= 1
    assert w.cost_scale < 0  # C / max C
    for v, n in ((w.r, w.n), (w.c, w.m)):
        _marginal_ok(v, n)
        assert v.max() / v.min() <= 10.0 + 1e-9  # U(0.1, 1) draws, normalised


def test_image_grid():
    w = W.image_grid()
    assert (w.n, w.m, w.eta, w.tol) == (4096, 4096, 1e-3, 1e-6)
    C = w.C
    assert C.shape == (4096, 4096) and C.dtype == np.float32 and C.nbytes == 64 * 2 ** 20
    assert C.min() == 0.0 and C.max() == 1.0 and np.all(np.diag(C) == 0.0)
    assert np.array_equal(C, C.T)
    # squared grid distance / max: neighbours on the 64 x 64 unit grid are 1 / (2 * 63^2) apart
    assert C[0, 1] == pytest.approx(1.0 / (2 * 63 ** 2), rel=1e-6)
    for v in (w.r, w.c):
        _marginal_ok(v, 4096)
        assert v.min() >= 1e-6 / (1 + 4096 * 1e-6) * 0.99  # floor 1e-6 before renormalising


def test_highdim():
    w = W.highdim()
    assert (w.n, w.m, w.d, w.eta, w.tol, w.cost_scale) == (1 << 15, 1 << 15, 64, 0.0, 1e-6, 1.0)
    assert abs(float(w.x.mean())) < 0.01 and abs(float(w.y.mean()) - 0.5) < 0.01
    assert abs(float(w.x.std()) - 1.0) < 0.01 and abs(float(w.y.std()) - 1.0) < 0.01
    for v in (w.r, w.c):
        _marginal_ok(v, 1 << 15)
        assert np.ptp(v) == 0.0  # uniform


def test_diffloss():
    w = W.diffloss()
    assert (w.n, w.m, w.d, w.eta, w.tol) == (8192, 8192, 3, 1e-2, 1e-6)
    assert abs(float(w.x.mean())) < 0.05 and abs(float(w.x.std()) - 1.0) < 0.05
    norms = np.linalg.norm(w.y.astype(np.float64), axis=1)
    assert abs(norms.mean() - 1.0) < 0.01 and norms.std() < 0.1  # unit sphere + N(0, 0.05^2)
    for v in (w.r, w.c):
        _marginal_ok(v, 8192)


def test_largescale():
    w = W.largescale()
    assert (w.n, w.m, w.d, w.eta, w.tol) == (1 << 18, 1 << 18, 3, 0.0, 1e-5)
    assert w.x.min() >= 0 and w.x.max() <= 1 and w.y.min() >= 0 and w.y.max() <= 1
    assert abs(float(w.x.mean()) - 0.5) < 0.01
    for v, n in ((w.r, w.n), (w.c, w.m)):
        _marginal_ok(v, n)
        assert v.max() / v.min() <= 10.0 + 1e-9


@pytest.mark.parametrize("gen", [W.plain_2d, W.diffloss, lambda: W.highdim(n=1024)])
def test_generators_are_deterministic(gen):
    a, b = gen(), gen()
    for k in ("x", "y", "r", "c"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
