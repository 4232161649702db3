"""Hybrid passes (half the feature columns recomputed, half streamed) vs the oracle.

Same tolerances as the stored and recompute paths (divergence 1e-4 relative,
residual 1e-5 absolute): every entry is either a stored shifted feature
exp(L - shift) or the recompute pass's ex2 of the expanded exponent, each
within the FP32 feature error the other parity tests allow. The shapes cover
every row-group width (ldr up to 256, 512 and 1024 give 1, 2 and 4 warps per
row), ragged r and ragged row counts (the last batch of a CTA partly past the
end), one point per cloud, and the smallest row stride the split allows (8).
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
    return prob, prob.values()


@pytest.mark.parametrize("debiased", [False, True])
@pytest.mark.parametrize("n,m,d,r,eps,iters", [
    (1, 1, 2, 8, 0.5, 3),
    (7, 5, 3, 5, 0.5, 20),          # ldr 8: one recomputed and one stored column group
    (33, 65, 2, 100, 0.3, 30),
    (1000, 777, 3, 128, 0.2, 40),
    (3001, 2999, 2, 256, 0.5, 25),
    (513, 1025, 16, 1024, 1.0, 15),
    (4099, 131, 3, 600, 0.4, 10),
    (2000, 3000, 5, 512, 0.3, 20),
    (5003, 4001, 3, 1021, 0.1, 30),  # ragged r at the largest width, the large workload's eps
    # r = 1024 with d <= 4 takes the update pass compiled for that stride:
    # ragged row counts, and clouds smaller than one batch (the stored rows past
    # the end are zero-filled in a ring slot that was never written)
    (5003, 4001, 3, 1024, 0.1, 30),
    (9, 3, 2, 1024, 0.5, 10),
    (1001, 999, 4, 1024, 0.3, 20),
])
def test_hybrid_matches_oracle(lsf, n, m, d, r, eps, iters, debiased):
    p = synth.small_problem(11 + n, n, m, d, r, eps, iters, weights="dirichlet")
    _, g = gpu(lsf, p, "hybrid", debiased)
    ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=debiased)
    assert g["status"] == 0
    assert abs(g["W_xy"] - ref["W_xy"]) <= 1e-4 * abs(ref["W_xy"]), (g["W_xy"], ref["W_xy"])
    assert abs(g["res_xy"] - ref["res_xy"]) <= 1e-5, (g["res_xy"], ref["res_xy"])
    if debiased:
        scale = abs(ref["W_xy"]) + 0.5 * abs(ref["W_xx"]) + 0.5 * abs(ref["W_yy"])
        assert abs(g["W_bar"] - ref["W_bar"]) <= 1e-4 * scale
        for k in ("res_xx", "res_yy"):
            assert abs(g[k] - ref[k]) <= 1e-5


def test_hybrid_stored_block_matches_oracle_features(lsf):
    # the stored block holds columns c0..ldr-1 of exp(L - shift), shift over all r
    p = synth.small_problem(5, 700, 10, 3, 1000, 0.2, 1)
    prob, _ = gpu(lsf, p, "hybrid", False)
    th = o.make_theta(p.X, p.Y, p.Z, p.eps)
    L = o.log_features(p.X, th.U, p.eps, th.q)
    sh = L.max(1)
    c0 = lsf.lsf_hybrid_columns(prob.theta.ldr)
    ref = np.zeros((p.n, prob.theta.ldr - c0))
    ref[:, : p.r - c0] = np.exp(L[:, c0:] - sh[:, None])
    Fs = prob.x.F.double().cpu().numpy()
    assert Fs.shape == ref.shape
    # the stored-feature tolerance of the other parity tests: (2 sqrt(d) + 4)
    # (|L| + |c|) 2^-24 on L and on the shift, twice that relative on F
    c = 0.75 * np.log(2 * th.q) - 0.5 * np.log(p.r) + (th.U ** 2).sum(1) / (p.eps * th.q)
    tolL = (2 * np.sqrt(3) + 4) * (np.abs(L) + np.abs(c)[None, :]) * 2.0 ** -24
    assert np.all(np.abs(prob.x.shift.double().cpu().numpy() - sh) <= tolL.max(axis=1) + 1e-6)
    tol = (2 * (tolL + tolL.max(axis=1)[:, None]) + 1e-6)[:, c0:]
    got = Fs[:, : p.r - c0]
    want = ref[:, : p.r - c0]
    assert np.all((np.abs(got - want) <= tol * want) | (np.abs(got - want) <= 1e-37))
    assert np.all(Fs[:, p.r - c0:] == 0.0)


def test_hybrid_agrees_with_stored_and_recompute_on_large_shape(lsf):
    p = synth.large_problem(seed=0, n=1 << 15, iters=50)
    _, gs = gpu(lsf, p, "stored", True)
    _, gh = gpu(lsf, p, "hybrid", True)
    _, gr = gpu(lsf, p, "recompute", True)
    scale = abs(gs["W_xy"]) + 0.5 * abs(gs["W_xx"]) + 0.5 * abs(gs["W_yy"])
    assert gh["status"] == 0
    assert abs(gh["W_bar"] - gs["W_bar"]) <= 1e-4 * scale
    assert abs(gh["W_bar"] - gr["W_bar"]) <= 1e-4 * scale
    assert abs(gh["W_xy"] - gs["W_xy"]) <= 1e-4 * abs(gs["W_xy"])


def test_hybrid_is_deterministic(lsf):
    p = synth.small_problem(9, 20000, 15000, 3, 1024, 0.1, 20)
    prob, g1 = gpu(lsf, p, "hybrid", True)
    prob.run(p.iters, debiased=True)
    g2 = prob.values()
    assert g1["W_bar"] == g2["W_bar"] and g1["res_xy"] == g2["res_xy"]


def test_hybrid_rejects_large_d_and_tiny_ldr(lsf):
    p = synth.small_problem(3, 50, 50, 20, 64, 0.5, 3)
    with pytest.raises(lsf.LsfError) as e:
        gpu(lsf, p, "hybrid", False)
    assert e.value.status == lsf.LSF_ERR_UNSUPPORTED
    p = synth.small_problem(3, 50, 50, 2, 3, 0.5, 3)      # r = 3: ldr 4 has no split
    with pytest.raises(lsf.LsfError) as e:
        gpu(lsf, p, "hybrid", False)
    assert e.value.status == lsf.LSF_ERR_UNSUPPORTED


def test_pipe_rate_probe(lsf):
    # the denominators of the recompute and hybrid rooflines: packed FMA near the
    # FP32 pipe's 128 lanes per clock per SM, ex2 near the special-function
    # unit's 32; the packed form is not slower than the scalar one
    r = lsf.lsf_probe_pipe_rates()
    assert 96.0 <= r["ffma2_lane_ops_per_clk_sm"] <= 132.0, r
    assert 64.0 <= r["ffma_lane_ops_per_clk_sm"] <= 132.0, r
    assert 16.0 <= r["ex2_per_clk_sm"] <= 33.0, r
    assert r["ffma2_lane_ops_per_clk_sm"] >= 0.95 * r["ffma_lane_ops_per_clk_sm"], r
