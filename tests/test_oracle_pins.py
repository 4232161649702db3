"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library
routine, a closed form, an identity from a proof, an invariant, an independent
optimiser, or brute force.  Together they are meant to catch a dropped term, a
wrong sign or index, or a transposed operand anywhere in the oracle.
"""
import math

import numpy as np
import pytest
import scipy.optimize
import scipy.special

from oracle import oracle as o
import synth


def _tiny_factors(seed=0, n=7, m=5, r=3, d=2, eps=0.5):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)) * 0.5
    Y = rng.standard_normal((m, d)) * 0.5 + 0.3
    Z = rng.standard_normal((r, d))
    a = rng.exponential(size=n); a /= a.sum()
    b = rng.exponential(size=m); b /= b.sum()
    th = o.make_theta(X, Y, Z, eps)
    Lx = o.log_features(X, th.U, eps, th.q)
    Ly = o.log_features(Y, th.U, eps, th.q)
    return X, Y, Z, a, b, th, Lx, Ly


# ---------------------------------------------------------------- Lambert W0

def test_lambert_w0_matches_scipy():
    z = np.concatenate([[0.0, 1e-300, 1e-12, math.e], np.logspace(-8, 12, 200)])
    w = o.lambert_w0(z)
    ref = scipy.special.lambertw(z, 0).real
    np.testing.assert_allclose(w, ref, rtol=2e-15, atol=1e-300)


def test_lambert_w0_special_values_and_identity():
    assert o.lambert_w0(0.0) == 0.0
    assert abs(o.lambert_w0(math.e) - 1.0) < 1e-15
    z = np.logspace(-6, 8, 57)
    w = o.lambert_w0(z)
    np.testing.assert_allclose(w * np.exp(w), z, rtol=1e-14)


# ---------------------------------------------------------------- Lemma 1 q, sigma

@pytest.mark.parametrize("R,eps,d", [(1.0, 0.5, 2), (1.73, 0.1, 3), (14.5, 1.0, 128), (3.0, 0.05, 16)])
def test_q_satisfies_lambert_characterisation(R, eps, d):
    # q = z/(2 W0(z)) with z = R^2/(eps d) means 2q = e^{W0(z)}, i.e. 2q log(2q) = z.
    q, sigma = o.gaussian_params(R, eps, d)
    z = R * R / (eps * d)
    assert abs(2 * q * math.log(2 * q) - z) <= 1e-13 * max(1.0, z)
    assert q > 0.5
    assert abs(sigma * sigma - q * eps / 4) <= 1e-15 * q * eps


def test_q_limit_small_radius():
    q0, _ = o.gaussian_params(0.0, 0.5, 2)
    q1, _ = o.gaussian_params(1e-6, 0.5, 2)
    assert q0 == 0.5 and abs(q1 - 0.5) < 1e-10


# ---------------------------------------------------------------- Lemma 1 R

def _norm(p):
    # one point's Euclidean norm by a plain loop over coordinates (brute force)
    return math.sqrt(math.fsum(float(c) * float(c) for c in p))


@pytest.mark.parametrize("far", ["x", "y"])
def test_radius_is_the_smallest_ball_holding_both_clouds(far):
    # Lemma 1 (Sec. 3.2) needs every point of both clouds in B(0, R); the
    # reading taken is the smallest such R centred at 0. So no point lies
    # outside, and some point of either cloud lies on the sphere. The farthest
    # point is planted once in X and once in Y, so a radius taken from one
    # cloud only fails one of the two cases.
    rng = np.random.default_rng(11)
    X = rng.standard_normal((37, 3)) * 0.5
    Y = rng.standard_normal((29, 3)) * 0.5 + 0.2
    target = X if far == "x" else Y
    target[17] = np.array([3.0, -4.0, 12.0])      # norm exactly 13
    R = o.radius(X, Y)
    norms = [_norm(p) for p in X] + [_norm(p) for p in Y]
    assert all(nv <= R * (1 + 1e-15) for nv in norms)
    assert abs(R - 13.0) <= 1e-14 * 13.0
    # symmetric in the two clouds; invariant to a rotation of both
    assert o.radius(Y, X) == R
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    assert abs(o.radius(X @ Q, Y @ Q) - 13.0) <= 1e-13


def test_radius_of_single_points_and_scaling():
    # one point per cloud: the larger of the two norms; a scaling c of both
    # clouds scales R by |c|
    assert o.radius(np.array([[0.6, 0.8]]), np.array([[0.0, 0.5]])) == pytest.approx(1.0, abs=1e-15)
    assert o.radius(np.array([[0.0, 0.5]]), np.array([[-0.6, -0.8]])) == pytest.approx(1.0, abs=1e-15)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((10, 5))
    Y = rng.standard_normal((8, 5))
    assert o.radius(-2.5 * X, -2.5 * Y) == pytest.approx(2.5 * o.radius(X, Y), rel=1e-15)


# ---------------------------------------------------------------- feature map

@pytest.mark.parametrize("d,eps", [(2, 0.5), (3, 0.1), (16, 1.0)])
def test_feature_product_identity_from_proof(d, eps):
    # Proof of Lemma 1: phi(x,u) phi(y,u) = (2q)^{d/2} k(x,y)
    #   exp(-4||u - (x+y)/2||^2/eps) exp(2||u||^2/(eps q)), pointwise in u.
    rng = np.random.default_rng(d)
    X = rng.standard_normal((9, d)) * 0.4
    Y = rng.standard_normal((9, d)) * 0.4
    q, sigma = o.gaussian_params(o.radius(X, Y), eps, d)
    U = sigma * rng.standard_normal((1, d))          # r = 1: phi_theta = phi
    lx = o.log_features(X, U, eps, q)[:, 0]
    ly = o.log_features(Y, U, eps, q)[:, 0]
    u = U[0]
    mid = 0.5 * (X + Y)
    rhs = (d / 2) * math.log(2 * q) - ((X - Y) ** 2).sum(1) / eps \
        - 4.0 * ((u - mid) ** 2).sum(1) / eps + 2.0 * (u @ u) / (eps * q)
    np.testing.assert_allclose(lx + ly, rhs, rtol=1e-13, atol=1e-12)


def test_features_scale_with_r():
    # phi_theta = r^{-1/2}(phi(x,u_1),...): duplicating every anchor halves each
    # squared entry, so k_theta is unchanged.
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 2)); Y = rng.standard_normal((5, 2))
    U = rng.standard_normal((6, 2)) * 0.3
    q = 0.9
    k1 = o.features(X, U, 0.5, q) @ o.features(Y, U, 0.5, q).T
    U2 = np.concatenate([U, U])
    k2 = o.features(X, U2, 0.5, q) @ o.features(Y, U2, 0.5, q).T
    np.testing.assert_allclose(k1, k2, rtol=1e-13)


def test_monte_carlo_unbiased_gaussian_kernel():
    # E_rho[phi(x,u) phi(y,u)] = k(x,y) for u ~ N(0, q eps/4 I) (Lemma 1).
    rng = np.random.default_rng(11)
    d, eps, r = 2, 0.5, 400_000
    X = rng.standard_normal((6, d)) * 0.4
    Y = rng.standard_normal((6, d)) * 0.4
    q, sigma = o.gaussian_params(o.radius(X, Y), eps, d)
    U = sigma * rng.standard_normal((r, d))
    Lx = o.log_features(X, U, eps, q) + 0.5 * math.log(r)   # per-anchor phi(x,u_k)
    Ly = o.log_features(Y, U, eps, q) + 0.5 * math.log(r)
    k = o.gaussian_kernel(X, Y, eps)
    for i in range(X.shape[0]):
        samples = np.exp(Lx[i][None, :] + Ly) / k[i][:, None]     # ratio per anchor, mean 1
        mean = samples.mean(axis=1)
        se = samples.std(axis=1) / math.sqrt(r)
        assert np.all(np.abs(mean - 1.0) < 6 * se + 1e-12), (mean, se)


def test_monte_carlo_rate_is_inverse_sqrt_r():
    # Prop. 3.2: the ratio error of k_theta vs k shrinks like r^{-1/2}.
    d, eps = 2, 1.0
    rng = np.random.default_rng(5)
    X = rng.standard_normal((5, d)) * 0.3
    Y = rng.standard_normal((5, d)) * 0.3
    q, sigma = o.gaussian_params(o.radius(X, Y), eps, d)
    k = o.gaussian_kernel(X, Y, eps)
    rs = [100, 1000, 10000, 100000]
    errs = []
    for r in rs:
        e = []
        for s in range(12):
            U = sigma * np.random.default_rng([r, s]).standard_normal((r, d))
            kt = o.features(X, U, eps, q) @ o.features(Y, U, eps, q).T
            e.append(np.sqrt(np.mean((kt / k - 1.0) ** 2)))
        errs.append(np.mean(e))
    slope = np.polyfit(np.log(rs), np.log(errs), 1)[0]
    assert -0.62 < slope < -0.38, (slope, errs)


# ---------------------------------------------------------------- Alg. 1

def test_factored_log_matches_dense_textbook():
    X, Y, Z, a, b, th, Lx, Ly = _tiny_factors()
    K = np.exp(Lx) @ np.exp(Ly).T                       # K_theta = xi^T zeta (Sec. 3.1)
    for iters in (1, 2, 7, 40):
        sd = o.sinkhorn_dense(K, a, b, iters)
        sl = o.sinkhorn_log(Lx, Ly, a, b, iters)
        np.testing.assert_allclose(sl["logu"], sd["logu"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(sl["logv"], sd["logv"], rtol=1e-12, atol=1e-12)
        assert abs(sl["residual"] - sd["residual"]) < 1e-13


def test_stopping_rule_stops_at_the_first_passing_check_of_the_dense_textbook():
    # the textbook solver on the explicit K gives the residual after every
    # iteration count; the stopped solve must end at the first multiple of k
    # whose residual is within tol, with that iteration's scalings
    X, Y, Z, a, b, th, Lx, Ly = _tiny_factors(seed=3, n=9, m=6, r=4)
    K = np.exp(Lx) @ np.exp(Ly).T
    res = {t: o.sinkhorn_dense(K, a, b, t)["residual"] for t in range(1, 61)}
    for k in (1, 3, 7):
        for tol in (1e-2, 1e-4, 1e-7):
            st = o.sinkhorn_log_tol(Lx, Ly, a, b, 60, tol, k)
            checks = [t for t in range(k, 61, k)] + ([] if 60 % k == 0 else [60])
            want = next((t for t in checks if res[t] <= tol), 60)
            assert st["iters"] == want, (k, tol, st["iters"], want)
            sd = o.sinkhorn_dense(K, a, b, want)
            np.testing.assert_allclose(st["logu"], sd["logu"], rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(st["logv"], sd["logv"], rtol=1e-12, atol=1e-12)
            assert abs(st["residual"] - res[want]) < 1e-13


def test_stopping_rule_on_a_rank_one_kernel_and_at_zero_tolerance():
    # one feature: K = xi zeta^T has rank one, so after one iteration
    # u o (K v) = a (sum b) = a exactly, and any positive tol stops at the first
    # check
    X, Y, Z, a, b, th, Lx, Ly = _tiny_factors(seed=5, n=8, m=6, r=1)
    st = o.sinkhorn_log_tol(Lx, Ly, a, b, 50, 1e-12, 1)
    assert st["iters"] == 1 and st["residual"] < 1e-14
    st = o.sinkhorn_log_tol(Lx, Ly, a, b, 50, 1e-12, 4)
    assert st["iters"] == 4
    # tol = 0 on a full-rank kernel is never met: the cap is reached
    X, Y, Z, a, b, th, Lx, Ly = _tiny_factors(seed=5, n=8, m=6, r=5)
    st = o.sinkhorn_log_tol(Lx, Ly, a, b, 13, 0.0, 5)
    assert st["iters"] == 13 and st["residual"] > 0.0


def test_scaled_matches_log():
    p = synth.tiny_problem(n=300, m=250, r=40, iters=30)
    th = o.make_theta(p.X, p.Y, p.Z, p.eps)
    Lx = o.log_features(p.X, th.U, p.eps, th.q)
    Ly = o.log_features(p.Y, th.U, p.eps, th.q)
    sl = o.sinkhorn_log(Lx, Ly, p.a, p.b, p.iters)
    ss = o.sinkhorn_scaled(Lx, Ly, p.a, p.b, p.iters)
    np.testing.assert_allclose(ss["logu"], sl["logu"], rtol=1e-11, atol=1e-10)
    np.testing.assert_allclose(ss["logv"], sl["logv"], rtol=1e-11, atol=1e-10)
    assert abs(ss["residual"] - sl["residual"]) < 1e-12


def test_mass_is_one_after_every_half_step():
    # Sec. 2: u^T K v = 1 whenever the loop has been applied once (weights sum to 1).
    *_, a, b, th, Lx, Ly = _tiny_factors(seed=2)
    s = o.sinkhorn_log(Lx, Ly, a, b, 15, track_mass=True)
    np.testing.assert_allclose(s["mass"], 1.0, rtol=1e-13)


def test_column_marginal_exact_after_v_half_and_rows_converge():
    *_, a, b, th, Lx, Ly = _tiny_factors(seed=4)
    K = np.exp(Lx) @ np.exp(Ly).T
    for iters, tol in ((3, None), (4000, 1e-12)):
        s = o.sinkhorn_log(Lx, Ly, a, b, iters)
        P = np.exp(s["logu"][:, None] + np.log(K) + s["logv"][None, :])
        np.testing.assert_allclose(P.sum(0), b, rtol=1e-12)          # v-half makes P^T 1 = b
        assert abs(np.abs(P.sum(1) - a).sum() - s["residual"]) < 1e-13
        if tol:
            assert s["residual"] < tol


def test_dual_estimate_equals_primal_and_dual_at_convergence():
    # Eq. (3) primal, Eq. (5) dual objective and Eq. (6) estimate coincide at the optimum.
    *_, a, b, th, Lx, Ly = _tiny_factors(seed=6)
    eps = th.eps
    logK = np.log(np.exp(Lx) @ np.exp(Ly).T)
    s = o.sinkhorn_log(Lx, Ly, a, b, 5000)
    w6 = o.dual_estimate(a, b, s["logu"], s["logv"], eps)
    w5 = o.dual_objective(a, b, s["logu"], s["logv"], logK, eps)
    w3 = o.primal_objective(s["logu"], s["logv"], logK, eps)
    assert abs(w6 - w5) < 1e-12 and abs(w6 - w3) < 1e-10


def test_dual_estimate_matches_independent_lbfgs_optimum():
    # Maximise the Eq. (5) objective directly with a generic optimiser.
    *_, a, b, th, Lx, Ly = _tiny_factors(seed=8)
    eps = th.eps
    K = np.exp(Lx) @ np.exp(Ly).T
    n, m = K.shape

    def negf(z):
        al, be = z[:n], z[n:]
        E = np.exp(al / eps)[:, None] * K * np.exp(be / eps)[None, :]
        f = a @ al + b @ be - eps * E.sum() + eps
        g = np.concatenate([a - E.sum(1), b - E.sum(0)])
        return -f, -g

    res = scipy.optimize.minimize(negf, np.zeros(n + m), jac=True, method="L-BFGS-B",
                                  options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 20000})
    s = o.sinkhorn_log(Lx, Ly, a, b, 5000)
    w = o.dual_estimate(a, b, s["logu"], s["logv"], eps)
    assert abs(-res.fun - w) < 1e-9 * max(1.0, abs(w))


def test_rank_one_closed_form():
    # r = 1: after one iteration P = a b^T and
    # W = eps [sum a log a - sum a log xi + sum b log b - sum b log zeta].
    rng = np.random.default_rng(9)
    Lx = rng.standard_normal((6, 1)); Ly = rng.standard_normal((4, 1))
    a = rng.exponential(size=6); a /= a.sum()
    b = rng.exponential(size=4); b /= b.sum()
    eps = 0.7
    s = o.sinkhorn_log(Lx, Ly, a, b, 1)
    w = o.dual_estimate(a, b, s["logu"], s["logv"], eps)
    closed = eps * (a @ np.log(a) - a @ Lx[:, 0] + b @ np.log(b) - b @ Ly[:, 0])
    assert abs(w - closed) < 1e-13
    assert s["residual"] < 1e-15


def test_single_point_gives_the_cost():
    # n = m = 1: W = -eps log k_theta(x, y) = c_theta(x, y) (Eq. 7).
    rng = np.random.default_rng(10)
    X = rng.standard_normal((1, 3)); Y = rng.standard_normal((1, 3))
    Z = rng.standard_normal((17, 3))
    eps = 0.8
    out = o.divergence(X, Y, np.ones(1), np.ones(1), Z, eps, iters=3, debiased=False)
    th = out["theta"]
    k = (o.features(X, th.U, eps, th.q) @ o.features(Y, th.U, eps, th.q).T)[0, 0]
    assert abs(out["W_xy"] - (-eps * math.log(k))) < 1e-12


def test_debiased_divergence_of_identical_measures_is_zero():
    p = synth.small_problem(1, 200, 200, 2, 30, 0.3, 20, weights="dirichlet")
    out = o.divergence(p.X, p.X.copy(), p.a, p.a.copy(), p.Z, p.eps, p.iters)
    assert abs(out["W_bar"]) < 1e-12 * (abs(out["W_xy"]) + 1)


def test_translation_moves_only_the_anchor_weights():
    # Moving points and anchors together leaves every ||p - u_k|| unchanged, so the
    # log-features change only through the per-anchor term ||u_k||^2/(eps q).
    p = synth.small_problem(2, 60, 70, 3, 20, 0.4, 25)
    th = o.make_theta(p.X, p.Y, p.Z, p.eps)
    shift = np.array([0.3, -1.1, 2.0])
    U2 = th.U + shift
    corr = ((U2 ** 2).sum(1) - (th.U ** 2).sum(1)) / (p.eps * th.q)
    for P in (p.X, p.Y):
        L = o.log_features(P, th.U, p.eps, th.q)
        L2 = o.log_features(P + shift, U2, p.eps, th.q)
        np.testing.assert_allclose(L2 - corr[None, :], L, rtol=1e-12, atol=1e-10)
    # the anchor weights do matter: moving the points alone (theta recomputed) changes W
    base = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=False)
    moved = o.divergence(p.X + 5.0, p.Y + 5.0, p.a, p.b, p.Z, p.eps, p.iters, debiased=False)
    assert abs(moved["W_xy"] - base["W_xy"]) > 1e-6


def test_permutation_invariance():
    p = synth.small_problem(3, 50, 40, 2, 25, 0.5, 30, weights="dirichlet")
    base = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters)
    pi = np.random.default_rng(0).permutation(p.n)
    pj = np.random.default_rng(1).permutation(p.m)
    perm = o.divergence(p.X[pi], p.Y[pj], p.a[pi], p.b[pj], p.Z, p.eps, p.iters)
    for key in ("W_xy", "W_xx", "W_yy", "W_bar"):
        assert abs(perm[key] - base[key]) < 1e-12 * max(1, abs(base[key]))


def test_kernel_approximation_improves_with_r():
    # Sec. 4 deviation D against dense Sinkhorn with the true Gaussian kernel.
    rng = np.random.default_rng(12)
    n, d, eps = 40, 2, 1.0
    X = rng.standard_normal((n, d)) * 0.5
    Y = rng.standard_normal((n, d)) * 0.3 + 0.5
    a = np.full(n, 1.0 / n); b = np.full(n, 1.0 / n)
    Kt = o.gaussian_kernel(X, Y, eps)
    sd = o.sinkhorn_dense(Kt, a, b, 500)
    rot = o.dual_estimate(a, b, sd["logu"], sd["logv"], eps)
    devs = {}
    for r in (30, 3000, 100000):
        ds = []
        for s in range(4):
            Z = np.random.default_rng([r, s]).standard_normal((r, d))
            out = o.divergence(X, Y, a, b, Z, eps, iters=500, debiased=False, mode="scaled")
            ds.append(abs(o.deviation(rot, out["W_xy"]) - 100.0))
        devs[r] = np.mean(ds)
    assert devs[100000] < devs[3000] < devs[30], devs
    assert devs[100000] < 1.0


# ---------------------------------------------------------------- gradient

def _fd_problem():
    rng = np.random.default_rng(13)
    n, m, d, r, eps = 6, 5, 2, 7, 0.5
    X = rng.standard_normal((n, d)) * 0.5
    Y = rng.standard_normal((m, d)) * 0.5 + 0.2
    Z = rng.standard_normal((r, d))
    a = rng.exponential(size=n); a /= a.sum()
    b = rng.exponential(size=m); b /= b.sum()
    th = o.make_theta(X, Y, Z, eps)
    return X, Y, a, b, th


@pytest.mark.parametrize("debiased", [False, True])
def test_envelope_gradient_matches_central_differences(debiased):
    X, Y, a, b, th = _fd_problem()
    iters = 1500
    key = "W_bar" if debiased else "W_xy"
    st = o.divergence(X, Y, a, b, theta=th, iters=iters, debiased=debiased)
    g = o.gradient(X, Y, a, b, th, st, debiased=debiased)["W_bar" if debiased else "W"]

    def W(X_, Y_, a_, b_):
        return o.divergence(X_, Y_, a_, b_, theta=th, iters=iters, debiased=debiased)[key]

    h = 1e-5
    for (name, arr) in (("X", X), ("Y", Y)):
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            e = np.zeros_like(arr); e[idx] = h
            args_p = [X, Y, a, b]; args_m = [X, Y, a, b]
            k = 0 if name == "X" else 1
            args_p[k] = arr + e; args_m[k] = arr - e
            fd[idx] = (W(*args_p) - W(*args_m)) / (2 * h)
        np.testing.assert_allclose(g[name], fd, rtol=1e-6, atol=1e-8)
    # weights: only zero-sum (simplex tangent) directions are meaningful; the
    # O(h^2) truncation error grows like 1/a_i^2, so use a smaller step here
    h = 2e-6
    for (name, w) in (("a", a), ("b", b)):
        for (i, j) in ((0, 1), (2, 4), (3, 0)):
            e = np.zeros_like(w); e[i] = h; e[j] = -h
            if name == "a":
                fd = (W(X, Y, a + e, b) - W(X, Y, a - e, b)) / (2 * h)
            else:
                fd = (W(X, Y, a, b + e) - W(X, Y, a, b - e)) / (2 * h)
            assert abs((g[name][i] - g[name][j]) - fd) < 1e-8 * max(1.0, abs(fd))


@pytest.mark.parametrize("debiased", [False, True])
def test_anchor_gradient_matches_central_differences(debiased):
    # q (and R) stay frozen; only the anchors move, as when U is learned.
    X, Y, a, b, th = _fd_problem()
    iters = 1500
    key = "W_bar" if debiased else "W_xy"
    st = o.divergence(X, Y, a, b, theta=th, iters=iters, debiased=debiased)
    g = o.anchor_gradient(X, Y, th, st, debiased=debiased)
    assert g.shape == th.U.shape

    def W(U_):
        t = o.Theta(th.q, th.sigma, U_, th.eps, th.R)
        return o.divergence(X, Y, a, b, theta=t, iters=iters, debiased=debiased)[key]

    h = 1e-5
    fd = np.zeros_like(th.U)
    for idx in np.ndindex(th.U.shape):
        e = np.zeros_like(th.U); e[idx] = h
        fd[idx] = (W(th.U + e) - W(th.U - e)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_joint_translation_gradient_is_the_anchor_weight_term():
    # Moving X, Y and U together by delta changes only ||u_k||^2/(eps q) (see the
    # translation pin above), so the directional derivative of W along a common
    # translation is the derivative of that term alone, computed here by central
    # differences of W with the points and anchors all moved.
    X, Y, a, b, th = _fd_problem()
    iters = 1500
    st = o.divergence(X, Y, a, b, theta=th, iters=iters, debiased=True)
    gp = o.gradient(X, Y, a, b, th, st, debiased=True)["W_bar"]
    gU = o.anchor_gradient(X, Y, th, st, debiased=True)
    total = gp["X"].sum(0) + gp["Y"].sum(0) + gU.sum(0)
    h = 1e-5
    for c in range(X.shape[1]):
        e = np.zeros(X.shape[1]); e[c] = h

        def W(s):
            t = o.Theta(th.q, th.sigma, th.U + s * e, th.eps, th.R)
            return o.divergence(X + s * e, Y + s * e, a, b, theta=t, iters=iters)["W_bar"]
        fd = (W(1.0) - W(-1.0)) / (2 * h)
        assert abs(total[c] - fd) < 1e-6 * max(1.0, abs(fd)), (c, total[c], fd)


# ---------------------------------------------------------------- arc-cosine features

@pytest.mark.parametrize("s", [0, 1, 2])
def test_arccos_closed_form_matches_monte_carlo(s):
    # k_s(x,y) = E_{u ~ N(0,I)} 2 max(0,u.x)^s max(0,u.y)^s, checked against the closed form
    rng = np.random.default_rng(20 + s)
    d = 3
    X = rng.standard_normal((4, d))
    Y = rng.standard_normal((3, d))
    Uz = rng.standard_normal((1_000_000, d))
    wx = np.maximum(Uz @ X.T, 0.0)
    wy = np.maximum(Uz @ Y.T, 0.0)
    if s == 0:
        wx, wy = (wx > 0).astype(float), (wy > 0).astype(float)
    else:
        wx, wy = wx ** s, wy ** s
    mc = 2.0 * (wx.T @ wy) / Uz.shape[0]
    np.testing.assert_allclose(mc, o.arccos_kernel(X, Y, s), rtol=0.03, atol=3e-3)


def test_arccos_special_values():
    x = np.array([[0.6, -0.8, 0.0]])
    assert abs(o.arccos_kernel(x, x, 0)[0, 0] - 1.0) < 1e-12          # angle 0: J_0 = pi
    assert abs(o.arccos_kernel(x, -x, 0)[0, 0]) < 1e-12               # angle pi
    assert abs(o.arccos_kernel(2 * x, x, 1)[0, 0] - 2.0) < 1e-12      # ||x|| ||y|| at angle 0
    y = np.array([[0.8, 0.6, 0.0]])                                    # orthogonal unit vectors
    assert abs(o.arccos_kernel(x, y, 1)[0, 0] - 1.0 / math.pi) < 1e-12
    assert abs(o.arccos_kernel(x, y, 0)[0, 0] - 0.5) < 1e-12


@pytest.mark.parametrize("s", [0, 1, 2])
def test_arccos_features_are_unbiased(s):
    # sum_k phi(x,u_k) phi(y,u_k) over r anchors u_k ~ N(0, sigma^2 I) -> k_s(x,y) + kappa
    rng = np.random.default_rng(30 + s)
    d, r, sigma, kappa = 2, 400_000, 1.5, 0.3
    X = rng.standard_normal((3, d)) * 0.7
    Y = rng.standard_normal((2, d)) * 0.7
    U = sigma * rng.standard_normal((r, d))
    Lx = o.arccos_log_features(X, U, s, sigma, kappa)
    Ly = o.arccos_log_features(Y, U, s, sigma, kappa)
    K = np.exp(Lx) @ np.exp(Ly).T
    np.testing.assert_allclose(K, o.arccos_kernel(X, Y, s) + kappa, rtol=0.03)


def test_arccos_kernel_is_bounded_below_by_kappa():
    rng = np.random.default_rng(40)
    U = 1.3 * rng.standard_normal((50, 4))
    X = rng.standard_normal((30, 4))
    Y = -X  # every projection changes sign: only the constant feature is shared
    K = np.exp(o.arccos_log_features(X, U, 1, 1.3, 0.2)) @ np.exp(o.arccos_log_features(Y, U, 1, 1.3, 0.2)).T
    assert np.all(K >= 0.2 * (1 - 1e-12))
    np.testing.assert_allclose(np.diag(K), 0.2, rtol=1e-12)


def test_arccos_factored_sinkhorn_matches_dense_textbook():
    rng = np.random.default_rng(41)
    n, m, d, r = 9, 7, 3, 20
    X = rng.standard_normal((n, d))
    Y = rng.standard_normal((m, d)) + 0.5
    a = rng.exponential(size=n); a /= a.sum()
    b = rng.exponential(size=m); b /= b.sum()
    U = 1.4 * rng.standard_normal((r, d))
    out = o.arccos_divergence(X, Y, a, b, U, 1, 1.4, 0.1, eps=1.0, iters=60, debiased=False)
    K = np.exp(o.arccos_log_features(X, U, 1, 1.4, 0.1)) @ np.exp(o.arccos_log_features(Y, U, 1, 1.4, 0.1)).T
    dense = o.sinkhorn_dense(K, a, b, 60)
    np.testing.assert_allclose(out["xy"]["logu"], dense["logu"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(out["W_xy"], o.dual_estimate(a, b, dense["logu"], dense["logv"], 1.0), rtol=1e-12)


# --------------------------------------------------------------------------
# Accelerated Sinkhorn (App. A.2, read as accelerated alternating minimisation)
# --------------------------------------------------------------------------

def _acc_case(seed, n, m, d, r, eps):
    p = synth.small_problem(seed, n, m, d, r, eps, 10, weights="dirichlet")
    th = o.make_theta(p.X, p.Y, p.Z, p.eps)
    return p, o.log_features(p.X, th.U, p.eps, th.q), o.log_features(p.Y, th.U, p.eps, th.q)


ACC_CASES = [(1, 60, 50, 2, 40, 0.5), (2, 80, 70, 3, 64, 0.1), (3, 100, 90, 2, 100, 0.05)]


@pytest.mark.parametrize("seed,n,m,d,r,eps", ACC_CASES)
def test_accelerated_reaches_the_sinkhorn_optimum(seed, n, m, d, r, eps):
    # both methods solve the same dual problem: the limit is the converged W of Alg. 1
    p, Lx, Ly = _acc_case(seed, n, m, d, r, eps)
    ref = o.sinkhorn_log(Lx, Ly, p.a, p.b, 4000)
    W_star = o.dual_estimate(p.a, p.b, ref["logu"], ref["logv"], eps)
    acc = o.sinkhorn_accelerated(Lx, Ly, p.a, p.b, 600)
    W = o.dual_estimate(p.a, p.b, acc["logu"], acc["logv"], eps)
    assert abs(W - W_star) <= 1e-7 * abs(W_star)
    assert acc["residual"] <= 1e-3
    # the reported value is Eq. (6) at a point whose plan has the mass of the
    # fitted marginal (1 up to the FP32 rounding of the stored weights)
    mass = max(abs(math.log(float(np.sum(p.a, dtype=np.float64)))),
               abs(math.log(float(np.sum(p.b, dtype=np.float64)))))
    assert abs(-eps * acc["phi"][-1] - W) <= eps * mass + 1e-12 * abs(W)


@pytest.mark.parametrize("seed,n,m,d,r,eps", ACC_CASES)
def test_accelerated_values_obey_duality_and_the_estimate_sequence_bound(seed, n, m, d, r, eps):
    # every accepted point is dual feasible: -eps phi <= W* (weak duality); and the
    # accelerated analysis gives phi(eta_k) - phi* <= ||eta* - eta_0||^2 / (2 A_k)
    # for the optimal point eta* nearest the start eta_0 = 0 (optimal points differ
    # by a shift (c, -c) of the two blocks)
    p, Lx, Ly = _acc_case(seed, n, m, d, r, eps)
    ref = o.sinkhorn_log(Lx, Ly, p.a, p.b, 4000)
    phi_star = o.dual_phi(Lx, Ly, p.a, p.b, ref["logu"], ref["logv"])
    e1, e2 = ref["logu"], ref["logv"]
    c = (e2.sum() - e1.sum()) / (len(e1) + len(e2))
    R2 = float(((e1 + c) ** 2).sum() + ((e2 - c) ** 2).sum())
    acc = o.sinkhorn_accelerated(Lx, Ly, p.a, p.b, 200)
    gaps = np.asarray(acc["phi"]) - phi_star
    assert np.all(gaps >= -1e-10)
    assert np.all(gaps <= R2 / (2.0 * np.asarray(acc["A"])))
    # A_k grows at least like k^2 / (8 L_max) when L never exceeds L_max
    k = np.arange(1, len(acc["A"]) + 1)
    assert np.all(np.asarray(acc["A"]) >= k ** 2 / (8.0 * max(acc["L"]) * 4.0))


def test_accelerated_single_point_is_the_closed_form():
    # n = m = 1: phi(eta) = log K for every eta, so W = -eps log K (Eq. 7) at once
    p, Lx, Ly = _acc_case(5, 1, 1, 2, 16, 0.3)
    logK = float(o.lse(Lx[0] + Ly[0], axis=0))
    acc = o.sinkhorn_accelerated(Lx, Ly, p.a, p.b, 5)
    W = o.dual_estimate(p.a, p.b, acc["logu"], acc["logv"], 0.3)
    assert abs(W - (-0.3 * logK)) <= 1e-12 * abs(logK)


def test_bf16_pair_split_precision():
    # the pair features of the tensor-core pass: hi + lo equals F to 2^-16
    # relative (a rounding to nearest bf16 is within 2^-8 of its argument,
    # relatively), and the rounding helper agrees with known bf16 values, ties
    # included
    from tests.bf16_split import bf16_value, rn_bf16_bits, split_pair
    assert rn_bf16_bits(np.array([1.0], np.float32))[0] == 0x3F80
    assert rn_bf16_bits(np.array([1.0 + 2.0 ** -8], np.float32))[0] == 0x3F80   # tie, to even
    assert rn_bf16_bits(np.array([1.0 + 3 * 2.0 ** -8], np.float32))[0] == 0x3F82  # tie, to even
    assert rn_bf16_bits(np.array([1.0 + 2.0 ** -8 + 2.0 ** -20], np.float32))[0] == 0x3F81
    rng = np.random.default_rng(3)
    F = np.exp(-rng.uniform(0.0, 80.0, size=200000)).astype(np.float32)
    hi, lo = split_pair(F)
    approx = bf16_value(hi).astype(np.float64) + bf16_value(lo).astype(np.float64)
    rel = np.abs(approx - F.astype(np.float64)) / F.astype(np.float64)
    assert rel.max() <= 2.0 ** -16
    assert (np.abs(bf16_value(hi).astype(np.float64) - F) / F).max() <= 2.0 ** -8
