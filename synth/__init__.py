"""Seeded synthetic inputs for the positive-feature Sinkhorn path.

This module only draws random numbers and arranges them into arrays; it holds
none of the method's arithmetic.  Both the FP64 oracle (through the tests) and
the CUDA path (through the tests and the benchmark) take their inputs from here,
so the two sides see the same FP32 values.

Everything is FP32 on output, since that is what the device path consumes; the
oracle widens the same FP32 values to FP64.

The anchors of the Gaussian feature map (Lemma 1) are drawn here as *standard*
normals ``Z`` (r x d).  Each side scales them by its own sigma; the random draw
itself is an input, not part of either implementation.

Workload shapes follow the paper's experiments (two Gaussian clouds in R^2 as in
Fig. 1, low-dimensional clouds, a 128-dimensional pair for differentiation).
The point sets of the paper's figures are not available as data, so every cloud
here is synthetic; see the recipes below.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem",
    "gmm_cloud",
    "tiny_problem",
    "large_problem",
    "diff_problem",
    "small_problem",
    "batched_problems",
    "serving_stream",
]


@dataclass
class Problem:
    """One divergence problem: two weighted clouds plus the anchor draw."""

    X: np.ndarray  # n x d float32
    Y: np.ndarray  # m x d float32
    a: np.ndarray  # n float32, positive
    b: np.ndarray  # m float32, positive
    Z: np.ndarray  # r x d float32, standard normal anchor draw
    eps: float
    iters: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def m(self) -> int:
        return int(self.Y.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    @property
    def r(self) -> int:
        return int(self.Z.shape[0])


def _f32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def gmm_cloud(rng: np.random.Generator, n: int, d: int, k: int = 3, std: float = 0.3,
              means: np.ndarray | None = None):
    """n draws from an equal-weight k-component isotropic Gaussian mixture.

    Means are standard normal in R^d unless given; returns (points, means).
    """
    if means is None:
        means = rng.standard_normal((k, d))
    comp = rng.integers(0, means.shape[0], size=n)
    pts = means[comp] + std * rng.standard_normal((n, d))
    return pts, means


def _uniform(n: int) -> np.ndarray:
    return np.full(n, 1.0 / n, dtype=np.float32)


def tiny_problem(seed: int = 0, n: int = 1000, m: int = 1000, d: int = 2, r: int = 100,
                 eps: float = 0.5, iters: int = 100) -> Problem:
    """Two 3-component mixtures in R^d (std 0.3); Y is the same mixture moved by +1.

    The +1 shift on every coordinate mirrors the (1,1) mean offset of the paper's
    two-Gaussian experiment in R^2.
    """
    rng = np.random.default_rng(seed)
    X, means = gmm_cloud(rng, n, d)
    Y, _ = gmm_cloud(rng, m, d, means=means)
    Y = Y + 1.0
    Z = rng.standard_normal((r, d))
    return Problem(_f32(X), _f32(Y), _uniform(n), _uniform(m), _f32(Z), eps, iters,
                   name=f"tiny n={n} m={m} d={d} r={r} eps={eps} iters={iters}")


def large_problem(seed: int = 0, n: int = 1 << 20, m: int | None = None, d: int = 3,
                  r: int = 1024, eps: float = 0.1, iters: int = 200) -> Problem:
    """X uniform on the unit cube, Y ~ N(0.5*1, 0.1^2 I), uniform weights."""
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    X = rng.random((n, d))
    Y = 0.5 + 0.1 * rng.standard_normal((m, d))
    Z = rng.standard_normal((r, d))
    return Problem(_f32(X), _f32(Y), _uniform(n), _uniform(m), _f32(Z), eps, iters,
                   name=f"large n={n} m={m} d={d} r={r} eps={eps} iters={iters}")


def diff_problem(seed: int = 0, n: int = 8192, m: int | None = None, d: int = 128,
                 r: int = 1024, eps: float = 1.0, iters: int = 50) -> Problem:
    """X ~ N(0, I_d), Y ~ N(mu, I_d) with mu a random direction of norm 1."""
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    mu = rng.standard_normal(d)
    mu = mu / np.linalg.norm(mu)
    Y = mu + rng.standard_normal((m, d))
    Z = rng.standard_normal((r, d))
    return Problem(_f32(X), _f32(Y), _uniform(n), _uniform(m), _f32(Z), eps, iters,
                   name=f"diff n={n} m={m} d={d} r={r} eps={eps} iters={iters}")


def small_problem(seed: int, n: int, m: int, d: int, r: int, eps: float, iters: int,
                  weights: str = "uniform", shift: float = 1.0) -> Problem:
    """Mixture clouds of arbitrary small shape for parity and edge-case tests.

    ``weights`` is "uniform" or "dirichlet" (Dirichlet(1), i.e. normalised
    exponentials).
    """
    rng = np.random.default_rng(seed)
    X, means = gmm_cloud(rng, n, d)
    Y, _ = gmm_cloud(rng, m, d, means=means)
    Y = Y + shift
    Z = rng.standard_normal((r, d))
    if weights == "dirichlet":
        a = rng.exponential(size=n)
        b = rng.exponential(size=m)
        a, b = a / a.sum(), b / b.sum()
    else:
        a, b = _uniform(n), _uniform(m)
    return Problem(_f32(X), _f32(Y), _f32(a), _f32(b), _f32(Z), eps, iters,
                   name=f"small n={n} m={m} d={d} r={r} eps={eps} iters={iters} w={weights}")


def _log_uniform_int(rng: np.random.Generator, lo: int, hi: int) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batched_problems(seed: int = 0, count: int = 512, iters: int = 100,
                     n_lo: int = 1 << 10, n_hi: int = 1 << 16) -> list[Problem]:
    """Independent problems of uneven shape; problem i is seeded by (seed, i).

    n, m log-uniform in [n_lo, n_hi]; d in {2, 3, 16}; r in {128, 256};
    eps log-uniform in [0.05, 1]; independent mixture clouds; Dirichlet(1) weights.
    """
    out = []
    for i in range(count):
        rng = np.random.default_rng([seed, i])
        n = _log_uniform_int(rng, n_lo, n_hi)
        m = _log_uniform_int(rng, n_lo, n_hi)
        d = int(rng.choice([2, 3, 16]))
        r = int(rng.choice([128, 256]))
        eps = float(math.exp(rng.uniform(math.log(0.05), math.log(1.0))))
        X, _ = gmm_cloud(rng, n, d)
        Y, _ = gmm_cloud(rng, m, d)
        a = rng.exponential(size=n)
        b = rng.exponential(size=m)
        Z = rng.standard_normal((r, d))
        out.append(Problem(_f32(X), _f32(Y), _f32(a / a.sum()), _f32(b / b.sum()), _f32(Z),
                           eps, iters, name=f"batched[{i}] n={n} m={m} d={d} r={r} eps={eps:.4g}"))
    return out


@dataclass
class Request:
    """One divergence request of a served stream."""

    arrival_s: float
    problem: Problem


def serving_stream(seed: int = 0, count: int = 10000, rate_per_s: float = 2000.0,
                   iters: int = 100, n_lo: int = 1 << 8, n_hi: int = 1 << 18,
                   materialize: bool = True) -> list[Request]:
    """Poisson arrivals of debiased-divergence requests of uneven shape.

    Inter-arrival times are exponential with mean 1/rate.  Sizes log-uniform in
    [n_lo, n_hi]; d in {2, 3, 16}; r in {128, 512}; eps in {0.05, 0.2, 1.0};
    mixture clouds; uniform weights.  With ``materialize=False`` the point
    arrays are left empty (shape only), which keeps a 10k-request schedule cheap.
    """
    rng = np.random.default_rng([seed, 7919])
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        prng = np.random.default_rng([seed, 7919, i])
        n = _log_uniform_int(prng, n_lo, n_hi)
        m = _log_uniform_int(prng, n_lo, n_hi)
        d = int(prng.choice([2, 3, 16]))
        r = int(prng.choice([128, 512]))
        eps = float(prng.choice([0.05, 0.2, 1.0]))
        if materialize:
            X, means = gmm_cloud(prng, n, d)
            Y, _ = gmm_cloud(prng, m, d)
            Z = prng.standard_normal((r, d))
        else:
            X = np.zeros((n, d)); Y = np.zeros((m, d)); Z = np.zeros((r, d))
        out.append(Request(t, Problem(_f32(X), _f32(Y), _uniform(n), _uniform(m), _f32(Z), eps,
                                      iters, name=f"req[{i}] n={n} m={m} d={d} r={r} eps={eps}")))
    return out
