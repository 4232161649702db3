"""Adjoint kernels vs the oracle's envelope gradient (Prop. 3.3), through the C-ABI.

The device and the oracle differentiate the same final iterate (same
iterations, same theta held fixed), so the comparison is direct. Tolerances:
relative error in the l2 norm of each gradient block 1e-4 (points, anchors);
elementwise 2e-4 (1 + |g|) for the weight gradients eps log u, which inherit the
potentials' error; and elementwise for the point and anchor gradients, so that a
wrong row cannot hide in the norm. An entry of those is a sum over features (or
points) of terms m * (p - u) whose features carry up to the stored-feature
tolerance of the parity tests, delta = 2 (2 sqrt(d) + 4)(|L| + |c|) 2^-24
relative; the entry may therefore differ from the oracle's by
1e-4 |g| + sum |term| delta + 1e-5 sum |term| (the last part for the rounding of
the r-vectors t), plus 1e4 * 2^-126: the device flushes terms below the FP32
normal range to zero, so an entry made of such terms (an anchor far from all
mass) may read 0 where the FP64 oracle keeps ~1e-40. A wrong row or a dropped
term is off by the size of the sum of |term|, far above that. The oracle's formula itself is pinned against
central differences at convergence in test_oracle_pins.py.
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
    ref["bounds"] = gradient_bounds(p, st, debiased)
    return prob, g, ref


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _feature_delta(L, th, d, r, eps):
    """Stored-feature relative tolerance per (point, feature) of the parity tests."""
    c = 0.25 * d * np.log(2 * th.q) - 0.5 * np.log(r) + (th.U ** 2).sum(1) / (eps * th.q)
    return 2 * (2 * np.sqrt(d) + 4) * (np.abs(L) + np.abs(c)[None, :]) * 2.0 ** -24


def _term_sums(P, U, L, logw, lt, delta, q=None):
    """Per entry: sum |term| and sum |term| delta, for the point gradient (q None:
    terms 4 m_ik (p_i - u_k) summed over k) or the anchor gradient (terms
    m_ik (4 (p_i - u_k) + 2 u_k / q) summed over i)."""
    M = np.exp(logw[:, None] + L + lt[None, :])
    if q is None:
        S = np.zeros_like(P)
        B = np.zeros_like(P)
    else:
        S = np.zeros_like(U)
        B = np.zeros_like(U)
    for i0 in range(0, P.shape[0], 32):
        A = 4 * np.abs(P[i0:i0 + 32, None, :] - U[None, :, :])
        if q is not None:
            A = A + 2 * np.abs(U)[None, :, :] / q
        Mi, Di = M[i0:i0 + 32], delta[i0:i0 + 32]
        if q is None:
            S[i0:i0 + 32] = np.einsum("ik,ikd->id", Mi, A)
            B[i0:i0 + 32] = np.einsum("ik,ikd->id", Mi * Di, A)
        else:
            S += np.einsum("ik,ikd->kd", Mi, A)
            B += np.einsum("ik,ikd->kd", Mi * Di, A)
    return S, B


def gradient_bounds(p, st, debiased, anchors=False):
    """(sum |term|, sum |term| delta) per entry of the point gradients (X, Y) or of
    the anchor gradient, from the oracle's final iterate; each term of Eq. (2)
    enters with its weight (1 or 1/2)."""
    th = st["theta"]
    X, Y = np.asarray(p.X, np.float64), np.asarray(p.Y, np.float64)
    Lx = o.log_features(X, th.U, p.eps, th.q)
    Ly = o.log_features(Y, th.U, p.eps, th.q)
    dx = _feature_delta(Lx, th, p.d, p.r, p.eps)
    dy = _feature_delta(Ly, th, p.d, p.r, p.eps)
    q = th.q if anchors else None
    parts = []  # (weight, side, P, L, delta, logw, lt)
    s = st["xy"]
    parts.append((1.0, "X", X, Lx, dx, s["logu"], o.lse(Ly + s["logv"][:, None], axis=0)))
    parts.append((1.0, "Y", Y, Ly, dy, s["logv"], o.lse(Lx + s["logu"][:, None], axis=0)))
    if debiased:
        for side, P, L, dl, key in (("X", X, Lx, dx, "xx"), ("Y", Y, Ly, dy, "yy")):
            t = st[key]
            parts.append((0.5, side, P, L, dl, t["logu"], o.lse(L + t["logv"][:, None], axis=0)))
            parts.append((0.5, side, P, L, dl, t["logv"], o.lse(L + t["logu"][:, None], axis=0)))
    out = {}
    for wgt, side, P, L, dl, lw, lt in parts:
        S, B = _term_sums(P, th.U, L, lw, lt, dl, q)
        key = "U" if anchors else side
        S0, B0 = out.get(key, (0.0, 0.0))
        out[key] = (S0 + wgt * S, B0 + wgt * B)
    return out


def check_elementwise(g, ref, bounds):
    """Every entry within 1e-4 |ref| + sum |term| delta + 1e-5 sum |term| + 1e4 * 2^-126."""
    S, B = bounds
    tol = 1e-4 * np.abs(ref) + B + 1e-5 * S + 1e4 * 2.0 ** -126
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
    check_elementwise(gX, ref["X"], ref["bounds"]["X"])
    check_elementwise(gY, ref["Y"], ref["bounds"]["Y"])
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
    check_elementwise(gU, ref, gradient_bounds(p, st, debiased, anchors=True)["U"])
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
