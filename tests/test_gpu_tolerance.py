"""Alg. 1's stopping rule on the GPU (lsf_solve_tol, lsf_debiased_tol) vs the oracle.

A solve with a tolerance ends at the first check (every k iterations, and at
the cap) where its residual ||u o (K v) - a||_1 is at most tol. The decision is
taken on the GPU's residual, which agrees with the oracle's to the parity
tolerance (1e-5 absolute), so the iteration count T it picks is checked for
what must hold, not for equality with the oracle's count: T is a multiple of k
(or the cap), the oracle's residual after T iterations is within tol + 1e-5,
and after T - k it is above tol - 1e-5; the divergence then matches the
oracle's after the same T iterations (1e-4 relative). A zero tolerance runs to
the cap and reproduces the fixed-count solve.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import oracle as o

pytestmark = pytest.mark.gpu

RES_ATOL = 1e-5
W_RTOL = 1e-4


@pytest.fixture(scope="module")
def lsf():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2006_07057_gb300 as m
    m.lib()
    return m


def problem(lsf, p, mode):
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
    return lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode=mode)


def oracle_factors(p):
    th = o.make_theta(p.X, p.Y, p.Z, p.eps)
    Lx = o.log_features(p.X, th.U, p.eps, th.q)
    Ly = o.log_features(p.Y, th.U, p.eps, th.q)
    return Lx, Ly


def check_stop(T, k, cap, tol, res_at):
    """T iterations were run by a solve stopped with (tol, k, cap); res_at(t) is
    the oracle's residual after t iterations."""
    assert T == cap or T % k == 0, (T, k, cap)
    if T < cap:
        assert res_at(T) <= tol + RES_ATOL, (T, res_at(T), tol)
    if T > k:
        prev = T - k if T % k == 0 else T - T % k
        assert res_at(prev) > tol - RES_ATOL, (T, prev, res_at(prev), tol)


@pytest.mark.parametrize("mode", ["stored", "recompute", "hybrid", "log"])
@pytest.mark.parametrize("tol,k", [(1e-3, 5), (1e-4, 1), (2e-5, 7)])
def test_single_solve_stops_by_the_residual(lsf, mode, tol, k):
    p = synth.small_problem(31, 2000, 1500, 3, 128, 0.2, 0, weights="dirichlet")
    cap = 120
    prob = problem(lsf, p, mode)
    prob.run(cap, debiased=False, tol=tol, check_every=k)
    g = prob.values()
    assert g["status"] == 0
    T = g["iters"]
    Lx, Ly = oracle_factors(p)
    cache = {}

    def res_at(t):
        if t not in cache:
            cache[t] = o.sinkhorn_log(Lx, Ly, p.a, p.b, t)["residual"]
        return cache[t]

    check_stop(T, k, cap, tol, res_at)
    if T < cap:
        assert g["res_xy"] <= tol
    ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, T, debiased=False)
    assert abs(g["W_xy"] - ref["W_xy"]) <= W_RTOL * abs(ref["W_xy"]), (g["W_xy"], ref["W_xy"])
    assert abs(g["res_xy"] - ref["res_xy"]) <= RES_ATOL


@pytest.mark.parametrize("mode", ["stored", "hybrid", "log"])
def test_debiased_terms_stop_on_their_own(lsf, mode):
    # clouds of unequal spread: the three terms of Eq. (2) converge at different
    # rates, so their iteration counts differ
    p = synth.small_problem(37, 2500, 1800, 2, 96, 0.1, 0, weights="dirichlet")
    cap, tol, k = 150, 1e-4, 4
    prob = problem(lsf, p, mode)
    prob.run(cap, debiased=True, tol=tol, check_every=k)
    g = prob.values()
    assert g["status"] == 0
    Lx, Ly = oracle_factors(p)
    pairs = {"xy": (Lx, Ly, p.a, p.b), "xx": (Lx, Lx, p.a, p.a), "yy": (Ly, Ly, p.b, p.b)}
    W = {}
    for name, (L1, L2, w1, w2) in pairs.items():
        T = g["iters_" + name]
        cache = {}

        def res_at(t, L1=L1, L2=L2, w1=w1, w2=w2, cache=cache):
            if t not in cache:
                cache[t] = o.sinkhorn_log(L1, L2, w1, w2, t)["residual"]
            return cache[t]

        check_stop(T, k, cap, tol, res_at)
        st = o.sinkhorn_log(L1, L2, w1, w2, T)
        W[name] = o.dual_estimate(w1, w2, st["logu"], st["logv"], p.eps)
        assert abs(g["W_" + name] - W[name]) <= W_RTOL * abs(W[name]), (name, g["W_" + name], W[name])
        assert abs(g["res_" + name] - st["residual"]) <= RES_ATOL
    wbar = W["xy"] - 0.5 * (W["xx"] + W["yy"])
    scale = abs(W["xy"]) + 0.5 * abs(W["xx"]) + 0.5 * abs(W["yy"])
    assert abs(g["W_bar"] - wbar) <= W_RTOL * scale


@pytest.mark.parametrize("debiased", [False, True])
def test_zero_tolerance_runs_to_the_cap_like_the_fixed_count_solve(lsf, debiased):
    p = synth.small_problem(41, 3001, 2003, 3, 256, 0.3, 0, weights="dirichlet")
    lsf.lsf_set_small_solver(0)   # the same streamed passes on both sides
    try:
        a = problem(lsf, p, "stored")
        a.run(23, debiased=debiased, tol=0.0, check_every=5)
        ga = a.values()
        b = problem(lsf, p, "stored")
        b.run(23, debiased=debiased)
        gb = b.values()
    finally:
        lsf.lsf_set_small_solver(1)
    assert ga["iters"] == 23 and gb["iters"] == 23
    # the checks in between only read the state: the same passes, the same bits
    assert ga["W"] == gb["W"] and ga["res_xy"] == gb["res_xy"]
    if debiased:
        assert ga["iters_xx"] == ga["iters_yy"] == 23


def test_tolerance_arguments_are_checked(lsf):
    p = synth.small_problem(43, 50, 40, 2, 16, 0.5, 0)
    prob = problem(lsf, p, "stored")
    for kw in ({"tol": -1.0}, {"tol": float("nan")}, {"tol": 1e-3, "check_every": 0}):
        with pytest.raises(lsf.LsfError) as e:
            prob.run(10, debiased=False, **kw)
        assert e.value.status == lsf.LSF_ERR_ARG
    with pytest.raises(lsf.LsfError) as e:
        prob.run(0, debiased=True, tol=1e-3)
    assert e.value.status == lsf.LSF_ERR_ARG


def test_auto_mode_with_a_tolerance_picks_the_domain_and_stops(lsf):
    # LSF_MODE_AUTO with the stopping rule: the library builds the features,
    # picks the domain (the log domain after a range failure) and stops by the
    # residual; checked against the oracle after the iterations it ran
    for seed, d, eps, shift in ((51, 3, 0.3, 0.0), (17, 16, 0.05, 1.0)):
        p = synth.small_problem(seed, 400, 300, d, 128, eps, 0, weights="dirichlet", shift=shift)
        prob = problem(lsf, p, "auto")
        tol, k, cap = 1e-3, 5, 80
        prob.run(cap, debiased=False, tol=tol, check_every=k)
        g = prob.values()
        assert g["status"] == 0
        assert prob.used_mode in ("stored", "log")
        T = g["iters"]
        Lx, Ly = oracle_factors(p)
        cache = {}

        def res_at(t):
            if t not in cache:
                cache[t] = o.sinkhorn_log(Lx, Ly, p.a, p.b, t)["residual"]
            return cache[t]

        check_stop(T, k, cap, tol, res_at)
        ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, T, debiased=False)
        assert abs(g["W_xy"] - ref["W_xy"]) <= W_RTOL * abs(ref["W_xy"]), (seed, g["W_xy"], ref["W_xy"])
