"""Log-domain (stabilised) passes vs the oracle, through the C-ABI.

The oracle's primary solver is itself in the log domain (FP64), so it is valid
for every case here. Tolerances as for the scaling-domain path: divergence
1e-4 relative (debiased: relative to |W_xy| + |W_xx|/2 + |W_yy|/2), residual
1e-5 absolute. In the log domain the FP32 error of a feature entry is the
absolute error of L~ + log t, about |L| 2^-23 with |L| up to ~1000 nats for
d = 16, eps = 0.05; it enters W through a weighted average, so the same
relative tolerance holds. Each term of the residual sum |u s - a| carries that
error relative to u s, so for problems far from convergence (residual ~0.1-0.4
after 40 iterations at eps = 0.05) the residual bound is
1e-5 + 2 spread 2^-23 residual, spread the largest within-row log-feature range.
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


def check(g, ref, debiased, spread=0.0):
    assert g["status"] == 0, g["status"]
    assert abs(g["W_xy"] - ref["W_xy"]) <= 1e-4 * abs(ref["W_xy"]), (g["W_xy"], ref["W_xy"])
    rtol = 2.0 * spread * 2.0 ** -23
    assert abs(g["res_xy"] - ref["res_xy"]) <= 1e-5 + rtol * ref["res_xy"], (g["res_xy"], ref["res_xy"])
    if debiased:
        scale = abs(ref["W_xy"]) + 0.5 * abs(ref["W_xx"]) + 0.5 * abs(ref["W_yy"])
        assert abs(g["W_bar"] - ref["W_bar"]) <= 1e-4 * scale, (g["W_bar"], ref["W_bar"])
        for k in ("res_xx", "res_yy"):
            assert abs(g[k] - ref[k]) <= 1e-5 + rtol * ref[k], (k, g[k], ref[k])


@pytest.mark.parametrize("debiased", [False, True])
@pytest.mark.parametrize("n,m,d,r,eps,iters", [
    (1, 1, 2, 1, 0.5, 3),
    (7, 5, 3, 3, 0.5, 20),
    (33, 65, 2, 100, 0.3, 30),
    (1000, 777, 3, 128, 0.2, 40),
    (3001, 2999, 2, 256, 0.5, 25),
    (513, 1025, 16, 1024, 1.0, 15),
    (4099, 131, 3, 600, 0.4, 10),
])
def test_log_domain_matches_oracle(lsf, n, m, d, r, eps, iters, debiased):
    p = synth.small_problem(7 + n, n, m, d, r, eps, iters, weights="dirichlet")
    _, g = gpu(lsf, p, "log", debiased)
    ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=debiased)
    check(g, ref, debiased)


HARD = [(16, 0.05, 1.0, 17), (16, 0.05, 0.0, 18), (3, 0.05, 1.0, 19), (16, 0.1, 3.0, 20)]


@pytest.mark.parametrize("d,eps,shift,seed", HARD)
def test_log_domain_on_fp32_range_cases(lsf, d, eps, shift, seed):
    # log-feature spreads of 500-1000 nats: far outside the FP32 range of exp
    p = synth.small_problem(seed, 400, 300, d, 128, eps, 40, weights="dirichlet", shift=shift)
    ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=True)
    th = ref["theta"]
    spread = max(float(np.ptp(o.log_features(P, th.U, p.eps, th.q), axis=1).max()) for P in (p.X, p.Y))
    prob, g = gpu(lsf, p, "log", True)
    assert abs(float(prob.spread.item()) - spread) <= 1e-3 * spread
    check(g, ref, True, spread)
    # the scaling domain either matches or reports the failure; auto always matches
    _, gs = gpu(lsf, p, "stored", True)
    if gs["status"] == 0 and np.isfinite(gs["W_bar"]):
        pass
    else:
        assert gs["status"] & lsf.LSF_ERR_NONFINITE
    _, ga = gpu(lsf, p, "auto", True)
    check(ga, ref, True, spread)


def test_log_domain_gradient_matches_oracle(lsf):
    p = synth.small_problem(23, 600, 500, 3, 256, 0.2, 50, weights="dirichlet")
    prob, g = gpu(lsf, p, "log", True)
    assert g["status"] == 0
    gX, gY, ga, gb = [x.double().cpu().numpy() for x in prob.gradient()]
    st = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=True)
    ref = o.gradient(p.X, p.Y, p.a, p.b, st["theta"], st, debiased=True)["W_bar"]
    rel = lambda u, v: np.linalg.norm(u - v) / np.linalg.norm(v)  # noqa: E731
    assert rel(gX, ref["X"]) <= 1e-4 and rel(gY, ref["Y"]) <= 1e-4
    assert np.all(np.abs(ga - ref["a"]) <= 2e-4 * (1 + np.abs(ref["a"])))
    assert np.all(np.abs(gb - ref["b"]) <= 2e-4 * (1 + np.abs(ref["b"])))


def test_log_and_scaling_domains_agree(lsf):
    p = synth.large_problem(seed=0, n=1 << 14, iters=40)
    _, gs = gpu(lsf, p, "stored", True)
    _, gl = gpu(lsf, p, "log", True)
    scale = abs(gs["W_xy"]) + 0.5 * abs(gs["W_xx"]) + 0.5 * abs(gs["W_yy"])
    assert abs(gl["W_bar"] - gs["W_bar"]) <= 1e-4 * scale
