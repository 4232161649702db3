"""Batched persistent solver vs per-problem solves and the oracle (GPU).

Each problem of a batch is Alg. 1 on its own factored kernel; the batched
layouts (one persistent kernel over all tiles, or one thread-block cluster per
problem) only change how rows are scheduled and reduced, so its divergences must
match the oracle at the usual tolerances (1e-4 relative, residual 1e-5) and
agree with lsf_solve on the same problem. Cases cover fewer tiles than CTAs
(empty CTA ranges), many tiny problems straddling CTA boundaries, uneven n/m,
d and eps, both feature widths of the batched workload, and graph replay.
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsf():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2006_07057_gb300 as m
    m.lib()
    yield m
    m.lsf_set_batch_strategy(0)


@pytest.fixture(params=[0, 1], ids=["persistent", "clusters"])
def strategy(lsf, request):
    """Both layouts of a stored batch: one persistent kernel, or one cluster per problem."""
    lsf.lsf_set_batch_strategy(request.param)
    yield request.param
    lsf.lsf_set_batch_strategy(0)


class P:
    def __init__(self, p):
        c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        self.X, self.Y, self.a, self.b, self.Z = c(p.X), c(p.Y), c(p.a), c(p.b), c(p.Z)
        self.eps, self.iters, self.src = p.eps, p.iters, p


def make_batch(seed, count, n_lo, n_hi, r, iters, eps_lo=0.5):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        m = int(rng.integers(n_lo, n_hi + 1))
        d = int(rng.choice([2, 3, 16]))
        eps = float(math.exp(rng.uniform(math.log(eps_lo), 0.0)))
        out.append(synth.small_problem(1000 * seed + i, n, m, d, r, eps, iters, weights="dirichlet"))
    return out


def check_against_oracle(vals, probs):
    for v, p in zip(vals, probs):
        ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=False)
        assert v["status"] == 0, v
        assert abs(v["W"] - ref["W_xy"]) <= 1e-4 * abs(ref["W_xy"]), (v["W"], ref["W_xy"])
        assert abs(v["residual"] - ref["res_xy"]) <= 1e-5, (v["residual"], ref["res_xy"])


@pytest.mark.parametrize("seed,count,n_lo,n_hi,r", [
    (1, 3, 20, 60, 128),        # fewer tiles than CTAs
    (2, 40, 50, 3000, 128),
    (3, 25, 100, 5000, 256),
    (4, 200, 5, 80, 128),       # many tiny problems across CTA boundaries
])
def test_batched_matches_oracle(lsf, strategy, seed, count, n_lo, n_hi, r):
    probs = make_batch(seed, count, n_lo, n_hi, r, 25)
    solver = lsf.BatchedSolver([P(p) for p in probs], tile_bytes=32 * 1024)
    assert solver.info.strategy == strategy
    solver.run(25)
    check_against_oracle(solver.values(), probs)


def test_batched_agrees_with_single_solves(lsf, strategy):
    probs = make_batch(5, 12, 500, 20000, 256, 30)
    solver = lsf.BatchedSolver([P(p) for p in probs], tile_bytes=44 * 1024)
    solver.run(30)
    vals = solver.values()
    for v, p in zip(vals, probs):
        q = P(p)
        single = lsf.SinkhornProblem(q.X, q.Y, q.a, q.b, q.Z, p.eps)
        single.run(30, debiased=False)
        s = single.values()
        assert abs(v["W"] - s["W_xy"]) <= 1e-5 * abs(s["W_xy"]), (v["W"], s["W_xy"])
        assert abs(v["residual"] - s["res_xy"]) <= 1e-6


def test_batched_graph_replay_and_determinism(lsf, strategy):
    probs = make_batch(6, 30, 200, 4000, 128, 20)
    solver = lsf.BatchedSolver([P(p) for p in probs], tile_bytes=32 * 1024)
    solver.run(20)
    first = solver.values()
    solver.capture(20)
    solver.replay()
    torch.cuda.synchronize()
    again = solver.values()
    for x, y in zip(first, again):
        assert x["W"] == y["W"] and x["residual"] == y["residual"]


def test_range_failures_are_resolved_in_the_log_domain(lsf):
    # small eps with d = 16: some problems leave the FP32 range of the scaling domain
    probs = []
    for i, (d, eps) in enumerate([(16, 0.05), (3, 0.5), (16, 0.1), (2, 0.3), (16, 0.05)]):
        probs.append(synth.small_problem(300 + i, 300 + 50 * i, 250 + 40 * i, d, 128, eps, 30,
                                         weights="dirichlet", shift=2.0))
    solver = lsf.BatchedSolver([P(p) for p in probs], tile_bytes=32 * 1024, mode="auto")
    solver.run(30)
    vals = solver.values()
    for v, p in zip(vals, probs):
        ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=False)
        assert v["status"] == 0, v
        assert abs(v["W"] - ref["W_xy"]) <= 1e-4 * abs(ref["W_xy"]), (v["W"], ref["W_xy"])


def test_log_domain_batch_matches_oracle(lsf):
    probs = make_batch(8, 20, 100, 3000, 256, 25, eps_lo=0.05)
    solver = lsf.BatchedSolver([P(p) for p in probs], tile_bytes=32 * 1024, mode="log")
    solver.run(25)
    for v, p in zip(solver.values(), probs):
        ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=False)
        th = ref["theta"]
        spread = max(float(np.ptp(o.log_features(Q, th.U, p.eps, th.q), axis=1).max()) for Q in (p.X, p.Y))
        assert v["status"] == 0 and v["mode"] == "log"
        assert abs(v["W"] - ref["W_xy"]) <= 1e-4 * abs(ref["W_xy"]), (v["W"], ref["W_xy"])
        assert abs(v["residual"] - ref["res_xy"]) <= 1e-5 + 2 * spread * 2.0 ** -23 * ref["res_xy"]


def test_autotuner_picks_a_candidate(lsf):
    from paper_2006_07057_gb300 import autotune
    probs = make_batch(7, 10, 500, 3000, 128, 10)
    solver = lsf.BatchedSolver([P(p) for p in probs], tile_bytes=32 * 1024)
    tb = autotune.best_batch_tile(solver.batches[0][0], use_cache=False)
    assert tb in autotune.CANDIDATES
