"""Many weight vectors on one support (tensor-core pass) vs the FP64 oracle, through the C-ABI.

Each of the k weight pairs (a_p, b_p) on the same two clouds is solved by the
oracle on its own (Alg. 1 in the log domain from v = 1, Eq. (6)); the GPU solves
all k at once with the multi-right-hand-side pass. Tolerances: |W_gpu - W_orc|
<= 1e-4 |W_orc| and |res_gpu - res_orc| <= 1e-5, per pair.

The cases span ragged n and m (partial tiles of 64 points), r below and at a
multiple of 128 (zero feature padding), one to 20 right-hand sides (16 and 32
computed), and the single-point problem, whose divergence has the closed form
-eps log k_theta(x, y) (Eq. (7)) after any number of iterations.
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


def _weights(rng, k, n):
    W = rng.exponential(size=(k, n))
    return (W / W.sum(axis=1, keepdims=True)).astype(np.float32)


def _problem(seed, n, m, d, r, eps, k):
    p = synth.small_problem(seed, n, m, d, r, eps, 1)
    rng = np.random.default_rng(1000 + seed)
    return p, _weights(rng, k, n), _weights(rng, k, m)


def _oracle(p, A, B, iters):
    th = o.make_theta(p.X, p.Y, p.Z, p.eps)
    Lx = o.log_features(p.X, th.U, p.eps, th.q)
    Ly = o.log_features(p.Y, th.U, p.eps, th.q)
    out = []
    for a, b in zip(A, B):
        s = o.solve(Lx, Ly, a, b, iters)
        out.append({"W": o.dual_estimate(a, b, s["logu"], s["logv"], p.eps), "res": s["residual"]})
    return out


def _run(lsf, p, A, B, iters):
    dev = torch.device("cuda", 0)
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).to(dev) for k in "XYZ"}
    prob = lsf.MultiSinkhornProblem(t["X"], t["Y"], torch.from_numpy(A).to(dev),
                                    torch.from_numpy(B).to(dev), t["Z"], p.eps)
    prob.run(iters)
    return prob, prob.values()


@pytest.mark.parametrize("seed,n,m,d,r,eps,iters,k", [
    (31, 1000, 777, 2, 100, 0.5, 30, 5),
    (32, 3000, 2500, 3, 256, 0.2, 20, 16),
    (33, 700, 1500, 5, 300, 0.3, 15, 20),
    (34, 2048, 2048, 3, 1024, 0.1, 10, 8),
    (39, 1500, 1300, 3, 1024, 0.2, 12, 32),
    (40, 640, 900, 2, 896, 0.4, 10, 27),
    (35, 129, 300, 2, 64, 1.0, 25, 1),
])
def test_multi_matches_oracle(lsf, seed, n, m, d, r, eps, iters, k):
    p, A, B = _problem(seed, n, m, d, r, eps, k)
    ref = _oracle(p, A, B, iters)
    _, got = _run(lsf, p, A, B, iters)
    assert len(got) == k
    for q in range(k):
        g, e = got[q], ref[q]
        assert g["status"] == 0 and g["iters"] == iters
        assert abs(g["W"] - e["W"]) <= 1e-4 * abs(e["W"]), (q, g["W"], e["W"])
        assert abs(g["residual"] - e["res"]) <= 1e-5, (q, g["residual"], e["res"])


@pytest.mark.parametrize("seed,n,m,d,r,eps,iters,k", [
    (41, 900, 700, 2, 100, 0.3, 25, 6),
    (42, 1300, 1300, 3, 256, 0.5, 15, 17),
])
def test_multi_debiased_matches_oracle(lsf, seed, n, m, d, r, eps, iters, k):
    # Eq. (2) per pair: the self terms run on (X, X) with a_p and (Y, Y) with b_p,
    # all with the one theta of (X, Y)
    p, A, B = _problem(seed, n, m, d, r, eps, k)
    th = o.make_theta(p.X, p.Y, p.Z, p.eps)
    Lx = o.log_features(p.X, th.U, p.eps, th.q)
    Ly = o.log_features(p.Y, th.U, p.eps, th.q)
    dev = torch.device("cuda", 0)
    t = {q: torch.from_numpy(np.ascontiguousarray(getattr(p, q))).to(dev) for q in "XYZ"}
    prob = lsf.MultiSinkhornProblem(t["X"], t["Y"], torch.from_numpy(A).to(dev),
                                    torch.from_numpy(B).to(dev), t["Z"], p.eps)
    prob.run(iters, debiased=True)
    got = prob.values()
    for q in range(k):
        a, b = A[q], B[q]
        sxy = o.solve(Lx, Ly, a, b, iters)
        sxx = o.solve(Lx, Lx, a, a, iters)
        syy = o.solve(Ly, Ly, b, b, iters)
        Wxy = o.dual_estimate(a, b, sxy["logu"], sxy["logv"], p.eps)
        Wxx = o.dual_estimate(a, a, sxx["logu"], sxx["logv"], p.eps)
        Wyy = o.dual_estimate(b, b, syy["logu"], syy["logv"], p.eps)
        scale = abs(Wxy) + 0.5 * abs(Wxx) + 0.5 * abs(Wyy)
        g = got[q]
        assert g["status"] == 0
        assert abs(g["W_bar"] - (Wxy - 0.5 * (Wxx + Wyy))) <= 1e-4 * scale, (q, g["W_bar"])
        assert abs(g["W_xx"] - Wxx) <= 1e-4 * abs(Wxx) and abs(g["W_yy"] - Wyy) <= 1e-4 * abs(Wyy)
        assert abs(g["res_xx"] - sxx["residual"]) <= 1e-5 and abs(g["res_yy"] - syy["residual"]) <= 1e-5


def test_multi_resident_r_vectors_match_oracle(lsf):
    # the layout that keeps the split r-vectors in shared memory for the launch
    p, A, B = _problem(43, 1100, 900, 3, 256, 0.3, 9)
    ref = _oracle(p, A, B, 20)
    try:
        lsf.lsf_set_multi_tuning(0, 1, 1)
        _, got = _run(lsf, p, A, B, 20)
    finally:
        lsf.lsf_set_multi_tuning()
    for q in range(9):
        assert got[q]["status"] == 0
        assert abs(got[q]["W"] - ref[q]["W"]) <= 1e-4 * abs(ref[q]["W"])
        assert abs(got[q]["residual"] - ref[q]["res"]) <= 1e-5


def test_multi_flags_scalings_outside_fp32(lsf):
    # clouds 6 apart at eps = 0.01: every row product underflows in the scaling
    # domain, so each pair must report LSF_ERR_NONFINITE (as the single solve does)
    # rather than return a value
    p = synth.small_problem(44, 300, 280, 2, 64, 0.01, 1, shift=6.0)
    rng = np.random.default_rng(44)
    A, B = _weights(rng, 3, 300), _weights(rng, 3, 280)
    _, got = _run(lsf, p, A, B, 5)
    for g in got:
        assert g["status"] & lsf.LSF_ERR_NONFINITE, g
    dev = torch.device("cuda", 0)
    t = {q: torch.from_numpy(np.ascontiguousarray(getattr(p, q))).to(dev) for q in "XYZ"}
    single = lsf.SinkhornProblem(t["X"], t["Y"], torch.from_numpy(A[0]).to(dev),
                                 torch.from_numpy(B[0]).to(dev), t["Z"], p.eps, mode="stored")
    single.run(5, debiased=False)
    assert single.values()["status"] & lsf.LSF_ERR_NONFINITE


def test_split_features_bit_exact(lsf):
    # lsf_split_features against round-to-nearest-even done on the integer bits:
    # the same bf16 bit patterns for every entry, zeros in the padding columns
    from tests.bf16_split import split_pair
    p = synth.small_problem(45, 777, 10, 3, 200, 0.2, 1)
    dev = torch.device("cuda", 0)
    t = {q: torch.from_numpy(np.ascontiguousarray(getattr(p, q))).to(dev) for q in "XYZ"}
    R = float(lsf.lsf_radius(t["X"], t["Y"]).item())
    q_, sig = lsf.lsf_gaussian_params(R, p.eps, 3)
    U, c = lsf.lsf_anchors(t["Z"], q_, sig, p.eps)
    th = lsf.Theta(U, c, 200, lsf.ldr_for(200), 3, p.eps, R, q_, sig)
    F, _ = lsf.lsf_features(t["X"], th)
    F2 = lsf.lsf_split_features(F, 200, 256)
    torch.cuda.synchronize()
    got = F2.view(torch.int16).cpu().numpy().view(np.uint16)
    Fh = F.cpu().numpy()[:, :200]
    hi, lo = split_pair(Fh)
    assert np.array_equal(got[0, :, :200], hi) and np.array_equal(got[1, :, :200], lo)
    assert not got[:, :, 200:].any()


def test_multi_single_point_closed_form(lsf):
    # n = m = 1: P = a b^T after the first half steps and W = -eps log k_theta(x, y)
    p, A, B = _problem(36, 1, 1, 3, 50, 0.7, 3)
    th = o.make_theta(p.X, p.Y, p.Z, p.eps)
    Lx = o.log_features(p.X, th.U, p.eps, th.q)
    Ly = o.log_features(p.Y, th.U, p.eps, th.q)
    logk = float(o.lse(Lx[0] + Ly[0], axis=0))
    _, got = _run(lsf, p, A, B, 4)
    for g in got:
        assert g["status"] == 0
        assert abs(g["W"] - (-p.eps * logk)) <= 1e-4 * abs(p.eps * logk)
        assert g["residual"] <= 1e-6


def test_multi_each_pair_as_alone(lsf):
    # the same pair gives the same result alone (k = 1) and among 12 others
    p, A, B = _problem(37, 1500, 1200, 3, 200, 0.3, 13)
    _, mix = _run(lsf, p, A, B, 12)
    for q in (0, 6, 12):
        _, alone = _run(lsf, p, A[q:q + 1].copy(), B[q:q + 1].copy(), 12)
        assert abs(alone[0]["W"] - mix[q]["W"]) <= 1e-4 * abs(mix[q]["W"])
        assert abs(alone[0]["residual"] - mix[q]["residual"]) <= 1e-5


def test_multi_full_size_pairs_match_single_solves(lsf):
    # the bench's shape (n = m = 2^20 in R^3, r = 1024), 16 pairs, fewer iterations:
    # every pair against the stored-feature single solve of that pair, which is
    # itself held to the oracle at this size by the parity suite
    n = 1 << 20
    big = synth.large_problem(seed=0, n=n, iters=10)
    k = 16
    rng = np.random.default_rng(5)
    A = _weights(rng, k, n)
    B = _weights(rng, k, n)
    dev = torch.device("cuda", 0)
    t = {q: torch.from_numpy(getattr(big, q)).to(dev) for q in "XYZ"}
    tA, tB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    prob = lsf.MultiSinkhornProblem(t["X"], t["Y"], tA, tB, t["Z"], big.eps)
    prob.run(10)
    got = prob.values()
    for q in (0, 7, 15):
        single = lsf.SinkhornProblem(t["X"], t["Y"], tA[q].contiguous(), tB[q].contiguous(), t["Z"],
                                     big.eps, mode="stored")
        single.run(10, debiased=False)
        s = single.values()
        assert s["status"] == 0 and got[q]["status"] == 0
        assert abs(got[q]["W"] - s["W_xy"]) <= 1e-4 * abs(s["W_xy"]), (q, got[q]["W"], s["W_xy"])
        assert abs(got[q]["residual"] - s["res_xy"]) <= 1e-5, (q, got[q]["residual"], s["res_xy"])


def test_multi_rejects_unsupported_shapes(lsf):
    with pytest.raises(lsf.LsfError) as e:
        lsf.lsf_multi_workspace_bytes(128, 33)
    assert e.value.status == lsf.LSF_ERR_UNSUPPORTED
    with pytest.raises(lsf.LsfError) as e:
        lsf.lsf_multi_workspace_bytes(100, 4)
    assert e.value.status == lsf.LSF_ERR_UNSUPPORTED
    assert lsf.lsf_multi_workspace_bytes(1024, 32) > 0   # 4 x 32 + 32 x 8 = 384 TMEM columns
    p, A, B = _problem(38, 300, 200, 2, 64, 0.5, 3)
    prob, _ = _run(lsf, p, A, B, 2)
    small = prob.workspace[:1024]
    with pytest.raises(lsf.LsfError) as e:
        lsf.lsf_solve_multi(prob.theta, prob.ldr2, prob.F2x, prob.shift_x, prob.A, prob.F2y,
                            prob.shift_y, prob.B, 2, prob.U, prob.V, prob.Tu, prob.Tv,
                            prob.results, small)
    assert e.value.status == lsf.LSF_ERR_WORKSPACE
