"""Arc-cosine positive features (Sec. 3.2 and its appendix lemma) on the device vs the oracle.

Features: the log-features c_k + s log(u_k.x) (exact zeros where u_k.x <= 0) and
the merged constant feature log sqrt(kappa) are checked against the FP64 oracle;
the projection u.x is an FP32 dot product of d terms, so the log-feature error is
about s (d + 4) 2^-24 |u||x| / |u.x|, allowed with a floor for projections near 0
(those features are tiny after the row shift). The solves (stored, log domain,
multi-launch and cluster paths) then use the tolerances of the Gaussian parity
tests: 1e-4 relative on the divergences, 1e-5 absolute on the residual.
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


def dev(p):
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    return c(p.X), c(p.Y), c(p.a), c(p.b), c(p.Z)


@pytest.mark.parametrize("s", [0, 1, 2])
@pytest.mark.parametrize("n,d,r", [(300, 3, 100), (257, 16, 255), (129, 48, 511)])
def test_arccos_features_match_oracle(lsf, s, n, d, r):
    p = synth.small_problem(3 + s, n, n, d, r, 1.0, 1)
    sigma, kappa = 1.5, 0.2
    X, Y, a, b, Z = dev(p)
    prob = lsf.SinkhornProblem(X, Y, a, b, Z, 1.0, kernel="arccos", s=s, sigma=sigma, kappa=kappa)
    U = sigma * np.asarray(p.Z, np.float64)          # the oracle's own anchors
    L = o.arccos_log_features(p.X, U, s, sigma, kappa)
    shift = L.max(axis=1)
    F = prob.x.F.double().cpu().numpy()
    ldr = prob.arccos.ldr
    assert F.shape == (n, ldr) and np.all(F[:, r + 1:] == 0.0)
    ref = np.exp(L - shift[:, None])
    # FP32 projection: |dw| <= (d + 2) 2^-24 sum_d |x_d u_d| (accumulation and the
    # rounding of u = sigma z); L = c + s log w then carries s |dw| / w, and c,
    # log and the shift a few roundings of |L|
    Xd = np.asarray(p.X, np.float64)
    w = Xd @ U.T
    scale = np.abs(Xd) @ np.abs(U.T)
    dw = (d + 2) * 2.0 ** -24 * scale
    sure = np.abs(w) > dw                              # the sign of u.x is certain
    assert np.all(F[:, :r][sure & (w <= 0)] == 0.0)    # exact zeros
    tolL = np.zeros_like(L)
    tolL[:, :r] = s * dw / np.maximum(np.abs(w), 1e-300)
    tolL += 8 * 2.0 ** -24 * np.where(np.isfinite(L), np.abs(L), 0.0)
    row = tolL[np.arange(n), L.argmax(axis=1)]        # error of the shift
    check = np.isfinite(L)
    check[:, :r] &= sure & (tolL[:, :r] < 1e-3)
    bound = ref * np.expm1(tolL + row[:, None]) + 1e-7
    err = np.abs(F[:, :r + 1] - ref)
    assert np.all(err[check] <= bound[check]), float((err - bound)[check].max())
    gshift = prob.x.shift.double().cpu().numpy()
    assert np.all(np.abs(gshift - shift) <= row + 1e-6 * (1 + np.abs(shift)))


@pytest.mark.parametrize("policy", [0, 2])
@pytest.mark.parametrize("s,mode", [(0, "stored"), (1, "stored"), (2, "stored"), (1, "log")])
def test_arccos_divergence_matches_oracle(lsf, s, mode, policy):
    lsf.lsf_set_small_solver(policy)
    try:
        p = synth.small_problem(60 + s, 700, 500, 3, 200, 1.0, 40, weights="dirichlet")
        sigma, kappa, eps = 1.4, 0.05, 0.7
        X, Y, a, b, Z = dev(p)
        prob = lsf.SinkhornProblem(X, Y, a, b, Z, eps, mode=mode, kernel="arccos", s=s,
                                   sigma=sigma, kappa=kappa)
        prob.run(p.iters, debiased=True)
        g = prob.values()
    finally:
        lsf.lsf_set_small_solver(1)
    U = sigma * np.asarray(p.Z, np.float64)          # the oracle's own anchors
    ref = o.arccos_divergence(p.X, p.Y, p.a, p.b, U, s, sigma, kappa, eps=eps, iters=p.iters)
    assert g["status"] == 0, g
    for k in ("W_xy", "W_xx", "W_yy"):
        assert abs(g[k] - ref[k]) <= 1e-4 * abs(ref[k]), (k, g[k], ref[k])
    assert abs(g["res_xy"] - ref["res_xy"]) <= 1e-5
    scale = abs(ref["W_xy"]) + 0.5 * abs(ref["W_xx"]) + 0.5 * abs(ref["W_yy"])
    assert abs(g["W_bar"] - ref["W_bar"]) <= 1e-4 * scale


def test_arccos_rejects_gaussian_only_paths(lsf):
    p = synth.small_problem(9, 50, 40, 2, 16, 1.0, 5)
    X, Y, a, b, Z = dev(p)
    with pytest.raises(ValueError):
        lsf.SinkhornProblem(X, Y, a, b, Z, 1.0, mode="recompute", kernel="arccos")
    prob = lsf.SinkhornProblem(X, Y, a, b, Z, 1.0, kernel="arccos")
    prob.run(5)
    with pytest.raises(NotImplementedError):
        prob.gradient()
    with pytest.raises(NotImplementedError):
        prob.anchor_gradient()
