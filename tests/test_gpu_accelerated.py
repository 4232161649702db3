"""Accelerated Sinkhorn (App. A.2) on the GPU vs the oracle, through the C-ABI.

The oracle (``sinkhorn_accelerated``, FP64) and the GPU driver (log-domain
passes, FP32 vectors, FP64 sums) take the same discrete decisions only where
those decisions are not ties at FP32 resolution: the block of larger gradient
norm and the line-search acceptance. The iterate-level cases below are chosen
with the oracle's decision margins far above FP32 rounding (the test asserts
it), and there both sides must agree on every decision (attempt count, final
L) and on W within 1e-4 relative. The residual reported here is the l1
gradient norm ||P 1 - a||_1 + ||P^T 1 - b||_1 at a point far from convergence;
the gradient-step sequence zeta grows (its steps a_k g have a_k ~ k^2/L), so
its FP32 entries carry rounding of |zeta| 2^-24 each update, accumulated like a
random walk over k updates, and the plan's marginals inherit it as a relative
error: |res_gpu - res_orc| <= 1e-5 + 2 sqrt(k) 2^-24 max(|zeta|, |eta|). At
convergence both reach the Alg. 1 optimum, whatever the decisions.
"""
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
    return m


def _tensors(p):
    return {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}


def _oracle_logs(p):
    th = o.make_theta(p.X, p.Y, p.Z, p.eps)
    return o.log_features(p.X, th.U, p.eps, th.q), o.log_features(p.Y, th.U, p.eps, th.q)


@pytest.mark.parametrize("seed,n,m,d,r,eps,iters", [
    (13, 1000, 800, 2, 256, 0.1, 40),
    (14, 300, 500, 5, 100, 0.3, 25),
    (15, 2000, 1500, 3, 200, 0.5, 20),
])
def test_accelerated_iterates_match_the_oracle(lsf, seed, n, m, d, r, eps, iters):
    p = synth.small_problem(seed, n, m, d, r, eps, iters, weights="dirichlet")
    Lx, Ly = _oracle_logs(p)
    ref = o.sinkhorn_accelerated(Lx, Ly, p.a, p.b, iters)
    # the decisions are far from ties (FP32 rounding of phi is ~1e-7 relative)
    assert ref["block_margin"] >= 1e-4 and ref["accept_margin"] >= 2e-5
    assert not ref["stopped"]
    t = _tensors(p)
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode="log")
    stats = prob.run_accelerated(iters, debiased=False)
    g = prob.values()
    assert g["status"] == 0
    assert stats[0]["iters"] == iters == g["iters"]
    assert stats[0]["attempts"] == sum(ref["attempts"])
    assert stats[0]["L"] == ref["L"][-1]
    W_ref = o.dual_estimate(p.a, p.b, ref["logu"], ref["logv"], p.eps)
    assert abs(g["W_xy"] - W_ref) <= 1e-4 * abs(W_ref), (g["W_xy"], W_ref)
    res_tol = 1e-5 + 2.0 * np.sqrt(iters) * 2.0 ** -24 * ref["vmax"]
    assert abs(g["res_xy"] - ref["residual"]) <= res_tol, (g["res_xy"], ref["residual"], res_tol)
    # log potentials: the same point up to FP32 rounding (compared where the weight is)
    lu, lv = prob.log_potentials("xy")
    pa, pb = p.a.astype(np.float64), p.b.astype(np.float64)
    assert np.abs((lu.cpu().numpy() - ref["logu"]) * pa).sum() <= 1e-4 * max(1.0, np.abs(ref["logu"] * pa).sum())
    assert np.abs((lv.cpu().numpy() - ref["logv"]) * pb).sum() <= 1e-4 * max(1.0, np.abs(ref["logv"] * pb).sum())


def test_accelerated_reaches_the_sinkhorn_optimum(lsf):
    p = synth.small_problem(21, 300, 250, 2, 128, 0.2, 300, weights="dirichlet")
    Lx, Ly = _oracle_logs(p)
    ref = o.sinkhorn_log(Lx, Ly, p.a, p.b, 4000)
    W_star = o.dual_estimate(p.a, p.b, ref["logu"], ref["logv"], p.eps)
    t = _tensors(p)
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode="log")
    stats = prob.run_accelerated(300, debiased=False)
    g = prob.values()
    assert g["status"] == 0
    # it may stop early once phi is stationary to FP32 rounding
    assert 1 <= stats[0]["iters"] <= 300
    assert abs(g["W_xy"] - W_star) <= 1e-4 * abs(W_star), (g["W_xy"], W_star, stats)
    assert g["res_xy"] <= 1e-2


def test_accelerated_debiased_divergence(lsf):
    # the self terms start at an exact tie of the block norms (the same data on
    # both sides): both implementations take block 1 there
    iters = 10
    p = synth.small_problem(15, 2000, 1500, 3, 200, 0.5, iters, weights="dirichlet")
    Lx, Ly = _oracle_logs(p)
    runs = {"xy": o.sinkhorn_accelerated(Lx, Ly, p.a, p.b, iters),
            "xx": o.sinkhorn_accelerated(Lx, Lx, p.a, p.a, iters),
            "yy": o.sinkhorn_accelerated(Ly, Ly, p.b, p.b, iters)}
    for rr in runs.values():
        assert rr["block_margin"] >= 1e-4 and rr["accept_margin"] >= 2e-5
    W = {k: o.dual_estimate(*((p.a, p.b) if k == "xy" else (p.a, p.a) if k == "xx" else (p.b, p.b)),
                            rr["logu"], rr["logv"], p.eps) for k, rr in runs.items()}
    W_bar = W["xy"] - 0.5 * (W["xx"] + W["yy"])
    t = _tensors(p)
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode="log")
    stats = prob.run_accelerated(iters, debiased=True)
    g = prob.values()
    assert [s_["attempts"] for s_ in stats] == [sum(runs[k]["attempts"]) for k in ("xy", "xx", "yy")]
    scale = abs(W["xy"]) + 0.5 * abs(W["xx"]) + 0.5 * abs(W["yy"])
    assert abs(g["W_bar"] - W_bar) <= 1e-4 * scale, (g["W_bar"], W_bar)


def test_accelerated_rejects_bad_arguments(lsf):
    p = synth.small_problem(3, 50, 40, 2, 16, 0.5, 3)
    t = _tensors(p)
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode="stored")
    with pytest.raises(ValueError):
        prob.run_accelerated(5)
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode="log")
    with pytest.raises(lsf.LsfError) as e:
        prob.run_accelerated(0)
    assert e.value.status == 1
    with pytest.raises(lsf.LsfError) as e:
        prob.run_accelerated(3, L0=-1.0)
    assert e.value.status == 1
