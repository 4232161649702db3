"""Adjoint kernels vs the oracle's envelope gradient (Prop. 3.3), through the C-ABI.

The device and the oracle differentiate the same final iterate (same
iterations, same theta held fixed), so the comparison is direct. Tolerances:
relative error in the l2 norm of each gradient block 1e-4 (points, anchors);
elementwise, every entry of a point or anchor gradient within
1e-4 (|g| + 1e-2 max|g|) of the oracle's (so that one wrong row cannot hide in
the norm; the floor covers entries that are sums of cancelling terms of the
block's typical size); and elementwise 2e-4 (1 + |g|) for the weight gradients
eps log u, which inherit the potentials' error. The oracle's formula itself is
pinned against central differences at convergence in test_oracle_pins.py.
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


def run_both(lsf, p, debiased):
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps)
    prob.run(p.iters, debiased=debiased)
    g = [x.double().cpu().numpy() for x in prob.gradient()]
    st = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=debiased)
    ref = o.gradient(p.X, p.Y, p.a, p.b, st["theta"], st, debiased=debiased)
    ref = ref["W_bar" if debiased else "W"]
    return prob, g, ref


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def check_elementwise(g, ref, rtol=1e-4, floor=1e-2):
    """Every entry within rtol (|ref| + floor max|ref|); reports the worst entry."""
    tol = rtol * (np.abs(ref) + floor * np.abs(ref).max())
    ratio = np.abs(g - ref) / tol
    worst = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    assert ratio[worst] <= 1.0, (f"entry {worst}: {g[worst]} vs {ref[worst]} "
                                 f"({ratio[worst]:.3g} x tolerance)")


@pytest.mark.parametrize("debiased", [False, True])
@pytest.mark.parametrize("n,m,d,r,eps,iters", [
    (1000, 1000, 2, 100, 0.5, 100),     # tiny workload shape
    (700, 900, 3, 256, 0.2, 60),
    (300, 257, 16, 1024, 1.0, 40),      # d = 16: warp-per-row kernel at its largest C
    (200, 190, 48, 512, 1.0, 30),       # d = 48: tiled contraction, partial column tile
    (1024, 1024, 128, 1024, 1.0, 50),   # differentiation workload shape at reduced n
])
def test_gradient_matches_oracle(lsf, n, m, d, r, eps, iters, debiased):
    if d == 128:
        p = synth.diff_problem(seed=0, n=n, iters=iters)
    else:
        p = synth.small_problem(31 + d, n, m, d, r, eps, iters, weights="dirichlet")
    prob, (gX, gY, ga, gb), ref = run_both(lsf, p, debiased)
    assert prob.values()["status"] == 0
    assert rel_l2(gX, ref["X"]) <= 1e-4, rel_l2(gX, ref["X"])
    assert rel_l2(gY, ref["Y"]) <= 1e-4, rel_l2(gY, ref["Y"])
    check_elementwise(gX, ref["X"])
    check_elementwise(gY, ref["Y"])
    assert np.all(np.abs(ga - ref["a"]) <= 2e-4 * (1 + np.abs(ref["a"])))
    assert np.all(np.abs(gb - ref["b"]) <= 2e-4 * (1 + np.abs(ref["b"])))


def test_autograd_function_matches_direct_gradient(lsf):
    p = synth.small_problem(41, 500, 400, 3, 128, 0.3, 40, weights="dirichlet")
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
    X = t["X"].clone().requires_grad_(True)
    Y = t["Y"].clone().requires_grad_(True)
    a = t["a"].clone().requires_grad_(True)
    b = t["b"].clone().requires_grad_(True)
    W = lsf.SinkhornDivergenceFn.apply(X, Y, a, b, t["Z"], p.eps, p.iters, True)
    (2.0 * W).backward()
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps)
    prob.run(p.iters, debiased=True)
    gX, gY, ga, gb = prob.gradient()
    assert abs(W.item() - prob.values()["W_bar"]) <= 1e-6 * abs(prob.values()["W_bar"]) + 1e-7
    torch.testing.assert_close(X.grad, 2.0 * gX)
    torch.testing.assert_close(Y.grad, 2.0 * gY)
    torch.testing.assert_close(a.grad, 2.0 * ga)
    torch.testing.assert_close(b.grad, 2.0 * gb)


# ---------------------------------------------------------------- anchors (theta gradient)

@pytest.mark.parametrize("debiased", [False, True])
@pytest.mark.parametrize("n,m,d,r,eps,iters,mode", [
    (1000, 1000, 2, 100, 0.5, 100, "stored"),   # tiny workload shape
    (700, 900, 3, 250, 0.2, 60, "stored"),      # ragged r (ldr 252), ragged rows
    (300, 257, 16, 1024, 1.0, 40, "stored"),    # two coordinate chunks of 8
    (200, 190, 48, 512, 1.0, 30, "stored"),
    (1024, 1024, 128, 1024, 1.0, 50, "stored"),  # differentiation workload shape at reduced n
    (600, 500, 3, 128, 0.3, 40, "log"),          # log-domain features and scalings
])
def test_anchor_gradient_matches_oracle(lsf, n, m, d, r, eps, iters, mode, debiased):
    if d == 128:
        p = synth.diff_problem(seed=0, n=n, iters=iters)
    else:
        p = synth.small_problem(51 + d, n, m, d, r, eps, iters, weights="dirichlet")
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode=mode)
    prob.run(p.iters, debiased=debiased)
    assert prob.values()["status"] == 0
    gU = prob.anchor_gradient().double().cpu().numpy()
    st = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=debiased)
    ref = o.anchor_gradient(p.X, p.Y, st["theta"], st, debiased=debiased)
    assert gU.shape == ref.shape
    assert rel_l2(gU, ref) <= 1e-4, rel_l2(gU, ref)
    check_elementwise(gU, ref)
    # deterministic: a second call gives the same bits
    gU2 = prob.anchor_gradient().double().cpu().numpy()
    assert np.array_equal(gU, gU2)


def test_anchor_gradient_wrt_draws_and_autograd(lsf):
    p = synth.small_problem(43, 500, 400, 3, 128, 0.3, 40, weights="dirichlet")
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
    Z = t["Z"].clone().requires_grad_(True)
    W = lsf.SinkhornDivergenceFn.apply(t["X"], t["Y"], t["a"], t["b"], Z, p.eps, p.iters, True)
    (3.0 * W).backward()
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps)
    prob.run(p.iters, debiased=True)
    gU = prob.anchor_gradient(wrt="U")
    gZ = prob.anchor_gradient(wrt="Z")
    sigma = prob.theta.sigma
    torch.testing.assert_close(gZ, sigma * gU, rtol=1e-6, atol=1e-7)
    torch.testing.assert_close(Z.grad, 3.0 * gZ)
    st = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=True)
    ref = sigma * o.anchor_gradient(p.X, p.Y, st["theta"], st, debiased=True)
    assert rel_l2(gZ.double().cpu().numpy(), ref) <= 1e-4
