"""Recompute-on-the-fly passes vs the oracle, and vs the stored-feature passes.

Same tolerances as the stored path (divergence 1e-4 relative, residual 1e-5
absolute): the recomputed entries come from the expanded exponent
A_k + B_i + x.W_k in FP32 and a hardware ex2, whose relative error per entry is
about |exponent| * 2^-23, the same order as the stored features'.
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


def gpu(lsf, p, mode, debiased):
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode=mode)
    prob.run(p.iters, debiased=debiased)
    return prob.values()


@pytest.mark.parametrize("debiased", [False, True])
@pytest.mark.parametrize("n,m,d,r,eps,iters", [
    (1, 1, 2, 1, 0.5, 3),
    (7, 5, 3, 3, 0.5, 20),
    (33, 65, 2, 100, 0.3, 30),
    (1000, 777, 3, 128, 0.2, 40),
    (3001, 2999, 2, 256, 0.5, 25),
    (513, 1025, 16, 1024, 1.0, 15),
    (4099, 131, 3, 600, 0.4, 10),
    (2000, 3000, 5, 512, 0.3, 20),
])
def test_recompute_matches_oracle(lsf, n, m, d, r, eps, iters, debiased):
    p = synth.small_problem(7 + n, n, m, d, r, eps, iters, weights="dirichlet")
    g = gpu(lsf, p, "recompute", debiased)
    ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=debiased)
    assert g["status"] == 0
    assert abs(g["W_xy"] - ref["W_xy"]) <= 1e-4 * abs(ref["W_xy"])
    assert abs(g["res_xy"] - ref["res_xy"]) <= 1e-5
    if debiased:
        scale = abs(ref["W_xy"]) + 0.5 * abs(ref["W_xx"]) + 0.5 * abs(ref["W_yy"])
        assert abs(g["W_bar"] - ref["W_bar"]) <= 1e-4 * scale
        for k in ("res_xx", "res_yy"):
            assert abs(g[k] - ref[k]) <= 1e-5


def test_recompute_agrees_with_stored_on_large_shape(lsf):
    p = synth.large_problem(seed=0, n=1 << 15, iters=50)
    gs = gpu(lsf, p, "stored", True)
    gr = gpu(lsf, p, "recompute", True)
    scale = abs(gs["W_xy"]) + 0.5 * abs(gs["W_xx"]) + 0.5 * abs(gs["W_yy"])
    assert abs(gr["W_bar"] - gs["W_bar"]) <= 1e-4 * scale
    assert abs(gr["W_xy"] - gs["W_xy"]) <= 1e-4 * abs(gs["W_xy"])


def test_recompute_rejects_large_d(lsf):
    p = synth.small_problem(3, 50, 50, 20, 64, 0.5, 3)
    with pytest.raises(lsf.LsfError) as e:
        gpu(lsf, p, "recompute", False)
    assert e.value.status == 32
