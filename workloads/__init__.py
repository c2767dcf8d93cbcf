"""Seeded synthetic inputs shared by the GPU path's tests/bench and the CPU oracle.

This module holds no arithmetic of the method (no cost normalisation, no LAMP
step): it only draws point clouds, stored cost matrices and marginals with the
shapes and distributions of the paper's workloads (Section 5 and App. E.2), so
that both sides of every parity check see identical arrays.

Every array is produced on the host with NumPy's PCG64 generator from a fixed
seed.  Point clouds and stored costs are float32 (the precision the GPU path
consumes); marginals are float64 and sum to one.

Workloads (sizes are the defaults; tests call the same recipes at smaller n, m):

* ``plain_2d``      n=m=256 points in [0,1]^2, r,c = normalised U(0.1,1) draws.
                    The cost is |x-y|^2 divided by its maximum (the solver's
                    cost_scale<0 option does the division).
* ``image_grid``    n=m=4096 supports of a 64x64 unit grid, stored dense cost =
                    squared grid distance normalised to max 1, marginals =
                    rasterised mixtures of 3-8 Gaussians + 1e-6 floor,
                    renormalised (App. E.2 support floor).  Stand-in for the
                    paper's 64x64 DOTmark images, which are not available.
* ``highdim``       n=m=2^15 points in R^64, x ~ N(0,I), y ~ N(0.5*1, I),
                    uniform marginals.
* ``diffloss``      n=m=8192 points in R^3, x ~ N(0,I), y = unit-sphere draws +
                    N(0, 0.05^2) noise, uniform marginals.
* ``largescale``    n=m=2^18 points in [0,1]^3, r,c = normalised U(0.1,1).
                    Stand-in for the paper's 512x512 colour-transfer run, whose
                    images are not available.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "Workload",
    "uniform_marginal",
    "random_marginal",
    "gaussian_mixture_marginal",
    "grid_points",
    "grid_sqdist_cost",
    "plain_2d",
    "image_grid",
    "highdim",
    "diffloss",
    "largescale",
    "points_problem",
    "dense_problem",
    "WORKLOADS",
    "bf16_round",
]


@dataclass
class Workload:
    """One synthetic problem instance.

    kind: "dense" (stored cost C given), or a point-cloud ground cost with points x, y
        given: "sqeuclid" (|x-y|^2), "l1", "linf" or "cosine".
    cost_scale: multiplier applied to |x-y|^2 by the solver; a negative value
        asks the solver to divide by the maximum cost (as in ``plain_2d``).
    eta, tol: entropic coefficient and L1 infeasibility target of the workload.
    """

    name: str
    kind: str
    n: int
    m: int
    d: int
    r: np.ndarray
    c: np.ndarray
    x: Optional[np.ndarray] = None
    y: Optional[np.ndarray] = None
    C: Optional[np.ndarray] = None
    cost_scale: float = 1.0
    eta: float = 0.0
    tol: float = 1e-6
    seed: int = 0
    notes: dict = field(default_factory=dict)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32:
    the points a bf16 tensor-core path actually multiplies."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(a))


def uniform_marginal(n: int) -> np.ndarray:
    return np.full(n, 1.0 / n, dtype=np.float64)


def random_marginal(rng: np.random.Generator, n: int, lo: float = 0.1, hi: float = 1.0) -> np.ndarray:
    v = rng.uniform(lo, hi, size=n).astype(np.float64)
    return v / v.sum()


def floor_and_renormalise(v: np.ndarray, floor: float = 1e-6) -> np.ndarray:
    """App. E.2 input preparation: add a small constant, then renormalise."""
    w = np.asarray(v, dtype=np.float64) + floor
    return w / w.sum()


def grid_points(side: int) -> np.ndarray:
    """Centres of a side x side grid on [0,1]^2, row-major, float32 (n = side^2)."""
    t = np.arange(side, dtype=np.float64) / max(side - 1, 1)
    gx, gy = np.meshgrid(t, t, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel()], axis=1).astype(np.float32)


def grid_sqdist_cost(side: int) -> np.ndarray:
    """Dense squared grid distance between the cells of a side x side grid,
    normalised so that its maximum is 1, stored float32 (n x n, row-major).

    On integer grid coordinates the maximum squared distance is 2(side-1)^2
    (App. D lists this value for the l2^2 DOTmark costs); dividing integer
    squared distances by it gives exact-as-possible float32 entries.
    """
    k = np.arange(side, dtype=np.int64)
    gi, gj = np.meshgrid(k, k, indexing="ij")
    pi = gi.ravel()
    pj = gj.ravel()
    d2 = (pi[:, None] - pi[None, :]) ** 2 + (pj[:, None] - pj[None, :]) ** 2
    return (d2.astype(np.float64) / float(2 * (side - 1) ** 2)).astype(np.float32)


def gaussian_mixture_marginal(rng: np.random.Generator, side: int, kmin: int = 3, kmax: int = 8) -> np.ndarray:
    """Rasterise a mixture of k ~ U{kmin..kmax} isotropic 2-D Gaussians on a
    side x side unit grid: means ~ U[0,1]^2, sigma ~ U(0.03, 0.2), weights ~
    Dirichlet(1).  Then apply the 1e-6 floor and renormalise."""
    k = int(rng.integers(kmin, kmax + 1))
    means = rng.uniform(0.0, 1.0, size=(k, 2))
    sig = rng.uniform(0.03, 0.2, size=k)
    wts = rng.dirichlet(np.ones(k))
    pts = grid_points(side).astype(np.float64)
    dens = np.zeros(pts.shape[0])
    for a in range(k):
        d2 = ((pts - means[a]) ** 2).sum(axis=1)
        dens += wts[a] * np.exp(-0.5 * d2 / sig[a] ** 2) / (2 * np.pi * sig[a] ** 2)
    dens /= dens.sum()
    return floor_and_renormalise(dens)


def points_problem(name: str, n: int, m: int, d: int, seed: int, dist: str = "uniform",
                   marg: str = "random", cost_scale: float = 1.0, eta: float = 0.0,
                   tol: float = 1e-6, grid_step: Optional[int] = None) -> Workload:
    """Generic point-cloud problem used by the named workloads and by tests
    at smaller / ragged sizes.

    dist: "uniform" (x, y ~ U[0,1]^d), "gauss_shift" (x ~ N(0,I), y ~ N(0.5,I)),
          "sphere" (x ~ N(0,I), y = unit-sphere + N(0,0.05^2)).
    marg: "random" (normalised U(0.1,1)) or "uniform".
    grid_step: if given, coordinates are rounded to multiples of 1/grid_step (a
        power of two keeps every squared distance exactly representable in float32).
    """
    rng = _rng(seed)
    if dist == "uniform":
        x = rng.uniform(0.0, 1.0, size=(n, d))
        y = rng.uniform(0.0, 1.0, size=(m, d))
    elif dist == "gauss_shift":
        x = rng.standard_normal(size=(n, d))
        y = rng.standard_normal(size=(m, d)) + 0.5
    elif dist == "sphere":
        x = rng.standard_normal(size=(n, d))
        g = rng.standard_normal(size=(m, d))
        y = g / np.linalg.norm(g, axis=1, keepdims=True) + 0.05 * rng.standard_normal(size=(m, d))
    else:
        raise ValueError(dist)
    if grid_step is not None:
        x = np.round(x * grid_step) / grid_step
        y = np.round(y * grid_step) / grid_step
    if marg == "random":
        r = random_marginal(rng, n)
        c = random_marginal(rng, m)
    elif marg == "uniform":
        r = uniform_marginal(n)
        c = uniform_marginal(m)
    else:
        raise ValueError(marg)
    return Workload(name=name, kind="sqeuclid", n=n, m=m, d=d, r=r, c=c,
                    x=np.ascontiguousarray(x, dtype=np.float32),
                    y=np.ascontiguousarray(y, dtype=np.float32),
                    cost_scale=cost_scale, eta=eta, tol=tol, seed=seed)


def half_norm_points(n: int, d: int, seed: int, nnz: int = 32) -> np.ndarray:
    """n points in R^d (d >= nnz) with nnz coordinates of +-1/8 at random positions and
    random signs, the rest 0: every coordinate is exact in bf16 and |x|^2 = nnz/64 exactly
    (1/2 for nnz = 32), so scaling to norm 1/sqrt(2) is exact (cosine-cost test points)."""
    rng = _rng(seed)
    x = np.zeros((n, d), np.float32)
    for i in range(n):
        idx = rng.choice(d, size=nnz, replace=False)
        x[i, idx] = np.where(rng.random(nnz) < 0.5, -0.125, 0.125).astype(np.float32)
    return x


def dense_problem(name: str, n: int, m: int, seed: int, eta: float = 0.0, tol: float = 1e-6,
                  marg: str = "random") -> Workload:
    """Random stored cost C ~ U[0,1) (float32, row-major n x m) with random marginals."""
    rng = _rng(seed)
    C = rng.uniform(0.0, 1.0, size=(n, m)).astype(np.float32)
    if marg == "random":
        r = random_marginal(rng, n)
        c = random_marginal(rng, m)
    else:
        r = uniform_marginal(n)
        c = uniform_marginal(m)
    return Workload(name=name, kind="dense", n=n, m=m, d=0, r=r, c=c, C=C,
                    eta=eta, tol=tol, seed=seed)


def plain_2d(n: int = 256, m: Optional[int] = None, seed: int = 11) -> Workload:
    m = n if m is None else m
    w = points_problem("plain_2d", n, m, 2, seed, dist="uniform", marg="random",
                       cost_scale=-1.0, eta=0.0, tol=1e-6)
    return w


def image_grid(side: int = 64, seed: int = 22) -> Workload:
    rng = _rng(seed)
    n = side * side
    C = grid_sqdist_cost(side)
    r = gaussian_mixture_marginal(rng, side)
    c = gaussian_mixture_marginal(rng, side)
    return Workload(name="image_grid", kind="dense", n=n, m=n, d=0, r=r, c=c, C=C,
                    eta=1e-3, tol=1e-6, seed=seed, notes={"side": side})


def highdim(n: int = 1 << 15, m: Optional[int] = None, d: int = 64, seed: int = 33) -> Workload:
    m = n if m is None else m
    return points_problem("highdim", n, m, d, seed, dist="gauss_shift", marg="uniform",
                          cost_scale=1.0, eta=0.0, tol=1e-6)


def diffloss(n: int = 8192, m: Optional[int] = None, seed: int = 44) -> Workload:
    m = n if m is None else m
    return points_problem("diffloss", n, m, 3, seed, dist="sphere", marg="uniform",
                          cost_scale=1.0, eta=1e-2, tol=1e-6)


def largescale(n: int = 1 << 18, m: Optional[int] = None, seed: int = 55) -> Workload:
    m = n if m is None else m
    return points_problem("largescale", n, m, 3, seed, dist="uniform", marg="random",
                          cost_scale=1.0, eta=0.0, tol=1e-5)


WORKLOADS = {
    "plain_2d": plain_2d,
    "image_grid": image_grid,
    "highdim": highdim,
    "diffloss": diffloss,
    "largescale": largescale,
}
