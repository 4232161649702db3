"""Cluster-persistent small-problem solver vs the multi-launch solver and the oracle.

Both solver paths run the same iterates of Alg. 1; the test forces each one
(lsf_set_small_solver policy 0 = multi-launch, 2 = cluster) on the same seeded
inputs and checks each against the FP64 oracle with the tolerances of the parity
tests (1e-4 relative on the divergences, 1e-5 absolute on the residual), then
checks that the cluster path is deterministic and that it also covers problems
whose rows do not fit in shared memory (read from L2 every half iteration).
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
    yield m
    m.lsf_set_small_solver(1)


def run(lsf, p, policy, debiased):
    lsf.lsf_set_small_solver(policy)
    try:
        t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
        prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps)
        lsf.lsf_launch_count_reset()
        prob.run(p.iters, debiased=debiased)
        vals = prob.values()
        vals["launches"] = lsf.lsf_launch_count()
        return prob, vals
    finally:
        lsf.lsf_set_small_solver(1)


def check(g, ref, debiased):
    assert g["status"] == 0, g
    assert abs(g["W_xy"] - ref["W_xy"]) <= 1e-4 * abs(ref["W_xy"]), (g["W_xy"], ref["W_xy"])
    assert abs(g["res_xy"] - ref["res_xy"]) <= 1e-5, (g["res_xy"], ref["res_xy"])
    if debiased:
        for k in ("W_xx", "W_yy"):
            assert abs(g[k] - ref[k]) <= 1e-4 * abs(ref[k]), (k, g[k], ref[k])
        for k in ("res_xx", "res_yy"):
            assert abs(g[k] - ref[k]) <= 1e-5, (k, g[k], ref[k])
        scale = abs(ref["W_xy"]) + 0.5 * abs(ref["W_xx"]) + 0.5 * abs(ref["W_yy"])
        assert abs(g["W_bar"] - ref["W_bar"]) <= 1e-4 * scale, (g["W_bar"], ref["W_bar"])


SHAPES = [
    (1, 1, 2, 1, 0.5, 3),          # one point each, r = 1
    (7, 5, 3, 3, 0.5, 20),         # fewer rows than CTAs of the cluster
    (1000, 1000, 2, 100, 0.5, 100),  # tiny workload shape
    (1000, 777, 3, 128, 0.2, 40),
    (513, 1025, 16, 1024, 1.0, 15),  # C = 8 columns per lane
    (3001, 2999, 2, 256, 0.5, 25),
]


@pytest.mark.parametrize("debiased", [False, True])
@pytest.mark.parametrize("n,m,d,r,eps,iters", SHAPES)
def test_both_paths_match_oracle(lsf, n, m, d, r, eps, iters, debiased):
    p = synth.small_problem(11 + n, n, m, d, r, eps, iters, weights="dirichlet")
    ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=debiased)
    _, g_multi = run(lsf, p, 0, debiased)
    _, g_small = run(lsf, p, 2, debiased)
    check(g_multi, ref, debiased)
    check(g_small, ref, debiased)
    # the cluster path is one solver launch (plus the Eq. (6) reduction and bookkeeping)
    assert g_small["launches"] < g_multi["launches"]


def test_cluster_path_is_deterministic(lsf):
    p = synth.small_problem(5, 900, 1100, 3, 256, 0.3, 30, weights="dirichlet")
    prob1, g1 = run(lsf, p, 2, True)
    prob2, g2 = run(lsf, p, 2, True)
    for k in ("W_xy", "W_xx", "W_yy", "W_bar", "res_xy"):
        assert g1[k] == g2[k], k
    assert torch.equal(prob1.s_xy.u, prob2.s_xy.u)
    assert torch.equal(prob1.s_xy.t_v, prob2.s_xy.t_v)


def test_rows_streamed_from_l2(lsf):
    # 6000 rows x 1024 features per cloud: a CTA's rows do not fit in shared memory
    p = synth.small_problem(6, 6000, 5000, 3, 1024, 0.5, 12)
    ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=True, mode="scaled")
    _, g = run(lsf, p, 2, True)
    check(g, ref, True)


def test_scalings_and_r_vectors_match_multi_launch(lsf):
    # the adjoint reads the final u~, v~ and t vectors: both paths must leave them alike
    p = synth.small_problem(8, 700, 600, 3, 200, 0.4, 25, weights="dirichlet")
    pa, _ = run(lsf, p, 0, True)
    pb, _ = run(lsf, p, 2, True)
    for s1, s2 in ((pa.s_xy, pb.s_xy), (pa.s_xx, pb.s_xx), (pa.s_yy, pb.s_yy)):
        for f in ("u", "v", "t_u", "t_v"):
            a, b = getattr(s1, f).double(), getattr(s2, f).double()
            assert torch.allclose(a, b, rtol=2e-4, atol=0), f
    ga = pa.gradient()
    gb = pb.gradient()
    for x, y in zip(ga, gb):
        assert torch.allclose(x, y, rtol=1e-3, atol=1e-6 * float(x.abs().max()))
