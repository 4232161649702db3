"""Plain FP64 CPU oracle for linear-time Sinkhorn with positive features.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the build
entry point and the CPU-baseline leg of the benchmark may import this module.
The product path (the CUDA library and its Python binding) never imports it and
shares no code with it.

What it computes, in the paper's order and notation (Scetbon & Cuturi,
"Linear Time Sinkhorn Divergences using Positive Features", arXiv 2006.07057):

* Lemma 1 (Sec. 3.2): the Gaussian kernel k(x,y) = exp(-||x-y||^2/eps) has the
  positive feature map
      phi(x,u) = (2q)^{d/4} exp(-2||x-u||^2/eps) exp(||u||^2/(eps q)),
  u ~ rho = N(0, sigma^2 I), sigma^2 = q eps / 4,
  q = R^2 / (2 eps d W0(R^2/(eps d))), W0 the principal Lambert branch.
  The Lemma statement prints the last exponent as ||u||^2/(eps(1/2 + R^2/eps));
  its proof derives ||u||^2/(eps q), the only form for which the integral
  identity holds (pinned by the Monte Carlo unbiasedness test).
* Sec. 3.2: phi_theta(x) = r^{-1/2} (phi(x,u_1), ..., phi(x,u_r)), u_k iid rho.
* Sec. 3.1: K_theta = xi^T zeta (here xi is stored point-major, n x r).
* Alg. 1 (Sec. 2): Sinkhorn scaling updates, run here as u <- a/(K v),
  v <- b/(K^T u) from v = 1 (one iteration = one u-half then one v-half); the
  reported residual is ||u o (K v) - a||_1 after the last v-half. With its
  stopping rule (``sinkhorn_log_tol``) the loop ends at the first test where
  that residual is at most the tolerance, tested every k iterations.
* Eq. (6): W_hat = eps (a^T log u + b^T log v).
* App. A.2: accelerated Sinkhorn, read as the accelerated alternating
  minimisation the appendix cites (its listing is garbled; see
  ``sinkhorn_accelerated``).
* Eq. (2): debiased W_bar = W(a,b) - (W(a,a) + W(b,b))/2 with one shared theta.
* Sec. 3.2 and its appendix lemma: the perturbed arc-cosine kernel k_s + kappa
  with features (sigma^{d/2} sqrt(2) max(0, u.x)^s exp(-||u||^2 (1 - 1/sigma^2)/4),
  sqrt(kappa)), u ~ N(0, sigma^2 I), sigma > 1.
* Prop. 3.3 and the formula after it (Sec. 3.3): dW/dK = -eps u v^T at the
  optimum, chained through xi(X) with theta held fixed; the same chain taken
  through the anchors U (q held fixed) gives the gradient a learned feature map
  needs (Sec. 3.3, learning the features).

The primary solver works in the log domain (always representable in FP64).
``sinkhorn_scaled`` runs the same iterates in the scaling domain with per-row
log shifts; it is faster and is checked against the log-domain solver.
``sinkhorn_dense`` is textbook Alg. 1 on an explicit matrix, for tiny inputs.

Every function here is pinned by tests against values fixed by the paper or the
mathematics (closed forms, invariants, library routines, brute force).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "lambert_w0",
    "gaussian_params",
    "radius",
    "anchors",
    "log_features",
    "features",
    "gaussian_kernel",
    "lse",
    "sinkhorn_log",
    "sinkhorn_scaled",
    "sinkhorn_dense",
    "dual_phi",
    "sinkhorn_accelerated",
    "dual_estimate",
    "dual_objective",
    "primal_objective",
    "Theta",
    "make_theta",
    "solve",
    "divergence",
    "gradient",
    "anchor_gradient",
    "arccos_kernel",
    "arccos_log_features",
    "arccos_divergence",
    "deviation",
]


# --------------------------------------------------------------------------
# Lemma 1 parameters
# --------------------------------------------------------------------------

def lambert_w0(z):
    """Principal branch W0 of the Lambert function for real z >= 0.

    W0(z) is the solution w >= 0 of w e^w = z (used by Lemma 1 to set q).
    Halley's iteration on f(w) = w e^w - z from the start w = log(1 + z), which
    lies above the root for z > 0; the iteration is run to FP64 convergence.
    """
    z = np.asarray(z, dtype=np.float64)
    if np.any(z < 0):
        raise ValueError("lambert_w0: this oracle only needs z >= 0")
    w = np.log1p(z)
    for _ in range(100):
        ew = np.exp(w)
        f = w * ew - z
        denom = ew * (w + 1.0) - (w + 2.0) * f / (2.0 * w + 2.0)
        step = np.where(denom != 0, f / np.where(denom != 0, denom, 1.0), 0.0)
        w_new = w - step
        done = np.all(np.abs(w_new - w) <= 4e-16 * np.maximum(np.abs(w_new), 1e-300))
        w = w_new
        if done:
            break
    return w if w.ndim else float(w)


def gaussian_params(R: float, eps: float, d: int) -> tuple[float, float]:
    """(q, sigma) of Lemma 1: q = R^2/(2 eps d W0(R^2/(eps d))), sigma^2 = q eps/4.

    As R -> 0, z/W0(z) -> 1 so q -> 1/2; that limit is returned for R = 0.
    """
    z = R * R / (eps * d)
    if z == 0.0:
        q = 0.5
    else:
        q = R * R / (2.0 * eps * d * lambert_w0(z))
    sigma = math.sqrt(q * eps / 4.0)
    return float(q), float(sigma)


def radius(X: np.ndarray, Y: np.ndarray) -> float:
    """R = largest Euclidean norm over both clouds, so that both lie in B(0, R).

    Lemma 1 asks for x, y in B(0, R) without saying how R is picked; this is the
    smallest such R centred at the origin.
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    rx = np.sqrt((X * X).sum(axis=1)).max() if X.shape[0] else 0.0
    ry = np.sqrt((Y * Y).sum(axis=1)).max() if Y.shape[0] else 0.0
    return float(max(rx, ry))


def anchors(Z: np.ndarray, sigma: float) -> np.ndarray:
    """Anchors u_k ~ N(0, sigma^2 I) from standard normal draws Z (r x d)."""
    return sigma * np.asarray(Z, dtype=np.float64)


# --------------------------------------------------------------------------
# Feature map
# --------------------------------------------------------------------------

def log_features(P: np.ndarray, U: np.ndarray, eps: float, q: float) -> np.ndarray:
    """log phi_theta(p)_k for every point p (rows of P) and anchor u_k (rows of U).

    log phi_theta(p)_k = (d/4) log(2q) - (1/2) log r - (2/eps)||p - u_k||^2
                         + ||u_k||^2/(eps q)
    (Lemma 1 feature with the proof's constant, scaled by r^{-1/2} as in the
    definition of phi_theta).  Returns an n x r FP64 array.
    """
    P = np.asarray(P, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    r, d = U.shape
    unorm2 = (U * U).sum(axis=1)
    const = (d / 4.0) * math.log(2.0 * q) - 0.5 * math.log(r)
    out = np.empty((P.shape[0], r))
    # rows are independent; they are processed in blocks only to bound memory
    step = max(1, (1 << 23) // max(1, r * d))
    for i0 in range(0, P.shape[0], step):
        diff = P[i0:i0 + step, None, :] - U[None, :, :]
        sq = (diff * diff).sum(axis=2)
        out[i0:i0 + step] = const - (2.0 / eps) * sq + unorm2[None, :] / (eps * q)
    return out


def features(P, U, eps, q):
    """phi_theta(p) for every row p of P, as an n x r array (may underflow)."""
    return np.exp(log_features(P, U, eps, q))


def gaussian_kernel(X, Y, eps):
    """k(x, y) = exp(-||x - y||^2 / eps), the kernel Lemma 1 decomposes."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    diff = X[:, None, :] - Y[None, :, :]
    return np.exp(-(diff * diff).sum(axis=2) / eps)


def lse(A: np.ndarray, axis: int) -> np.ndarray:
    """log sum exp along an axis, shifted by the maximum so nothing overflows."""
    mx = A.max(axis=axis, keepdims=True)
    mx = np.where(np.isfinite(mx), mx, 0.0)
    with np.errstate(divide="ignore"):  # an empty sum (all -inf) is log 0 = -inf
        out = np.log(np.exp(A - mx).sum(axis=axis, keepdims=True)) + mx
    return np.squeeze(out, axis=axis)


# --------------------------------------------------------------------------
# Alg. 1 on the factored kernel K = xi zeta^T
# --------------------------------------------------------------------------

def _log_Kv(Lx, Ly, logv):
    """log (K v) with K_ij = sum_k exp(Lx_ik + Ly_jk): first zeta^T v, then xi (.)."""
    lt = lse(Ly + logv[:, None], axis=0)          # log (zeta^T v)_k
    return lse(Lx + lt[None, :], axis=1), lt      # log (xi (zeta^T v))_i


def sinkhorn_log(Lx: np.ndarray, Ly: np.ndarray, a: np.ndarray, b: np.ndarray, iters: int,
                 track_mass: bool = False) -> dict:
    """Alg. 1 on K = exp(Lx) exp(Ly)^T in the log domain, FP64.

    Starts from v = 1 (log v = 0); each iteration is u <- a/(K v) then
    v <- b/(K^T u).  Returns log u, log v, the row residual ||u o (K v) - a||_1
    after the last v-half, and the two r-vectors t_u = log(xi^T u),
    t_v = log(zeta^T v) of the final state.  With ``track_mass`` the value
    u^T K v after every half step is recorded (it equals 1 after any update).
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    loga, logb = np.log(a), np.log(b)
    logu = np.zeros(Lx.shape[0])
    logv = np.zeros(Ly.shape[0])
    mass = []
    for _ in range(iters):
        logKv, _ = _log_Kv(Lx, Ly, logv)
        logu = loga - logKv
        if track_mass:
            mass.append(float(np.exp(lse(logu + logKv, axis=0))))
        logKtu, _ = _log_Kv(Ly, Lx, logu)
        logv = logb - logKtu
        if track_mass:
            mass.append(float(np.exp(lse(logv + logKtu, axis=0))))
    logKv, lt_v = _log_Kv(Lx, Ly, logv)
    residual = float(np.abs(np.exp(logu + logKv) - a).sum())
    lt_u = lse(Lx + logu[:, None], axis=0)
    return {"logu": logu, "logv": logv, "residual": residual, "lt_u": lt_u, "lt_v": lt_v,
            "mass": mass}


def sinkhorn_scaled(Lx: np.ndarray, Ly: np.ndarray, a: np.ndarray, b: np.ndarray,
                    iters: int) -> dict:
    """The same iterates as ``sinkhorn_log`` in the scaling domain, FP64.

    Rows are shifted by their maxima, xi~ = exp(Lx - mx), zeta~ = exp(Ly - my),
    so that K = diag(e^mx) xi~ zeta~^T diag(e^my); the shifted scalings
    u~ = u e^mx, v~ = v e^my then follow u~ = a/(xi~ (zeta~^T v~)),
    v~ = b/(zeta~ (xi~^T u~)).  v = 1 means v~ = e^my, stored as e^(my - M)
    with M = max my: a global factor that passes through every update
    (u~ carries e^M, v~ carries e^-M) and is removed when log u, log v are
    formed.  Valid while the FP64 range holds (row spread below ~700).
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    mx = Lx.max(axis=1)
    my = Ly.max(axis=1)
    Fx = np.exp(Lx - mx[:, None])
    Fy = np.exp(Ly - my[:, None])
    M = my.max()
    v = np.exp(my - M)
    u = np.zeros(Lx.shape[0])
    for _ in range(iters):
        u = a / (Fx @ (Fy.T @ v))
        v = b / (Fy @ (Fx.T @ u))
    s = Fx @ (Fy.T @ v)
    residual = float(np.abs(u * s - a).sum())
    logu = np.log(u) - mx - M
    logv = np.log(v) - my + M
    return {"logu": logu, "logv": logv, "residual": residual}


def sinkhorn_log_tol(Lx: np.ndarray, Ly: np.ndarray, a: np.ndarray, b: np.ndarray,
                     max_iters: int, tol: float, check_every: int = 1) -> dict:
    """Alg. 1 with its stopping rule (Sec. 2), in the log domain, FP64.

    The iterates of ``sinkhorn_log``; the loop ends at the first check where the
    row residual ||u o (K v) - a||_1 after the v-half is at most ``tol``.  The
    test is made after every ``check_every`` iterations and after
    ``max_iters`` at the latest (check_every = 1 is the algorithm as printed).
    Returns log u, log v, the last residual evaluated and the iterations run.
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    loga, logb = np.log(a), np.log(b)
    logu = np.zeros(Lx.shape[0])
    logv = np.zeros(Ly.shape[0])
    done = 0
    residual = math.inf
    while done < max_iters:
        for _ in range(min(check_every, max_iters - done)):
            logKv, _ = _log_Kv(Lx, Ly, logv)
            logu = loga - logKv
            logKtu, _ = _log_Kv(Ly, Lx, logu)
            logv = logb - logKtu
            done += 1
        logKv, _ = _log_Kv(Lx, Ly, logv)
        residual = float(np.abs(np.exp(logu + logKv) - a).sum())
        if residual <= tol:
            break
    return {"logu": logu, "logv": logv, "residual": residual, "iters": done}


def dual_phi(Lx, Ly, a, b, eta1, eta2) -> float:
    """phi(eta) = log <e^eta1, K e^eta2> - <eta1, a> - <eta2, b> (App. A.2, the dual
    of Eq. (5) in the coordinates eta = (alpha, beta)/eps, sign flipped so that it
    is minimised: W = -eps min phi)."""
    logKv, _ = _log_Kv(Lx, Ly, eta2)
    return float(lse(eta1 + logKv, axis=0) - eta1 @ a - eta2 @ b)


MAX_ATTEMPTS = 30  # line-search attempts per accelerated iteration before stopping


def sinkhorn_accelerated(Lx: np.ndarray, Ly: np.ndarray, a: np.ndarray, b: np.ndarray,
                         iters: int, L0: float = 1.0) -> dict:
    """Accelerated Sinkhorn (App. A.2) on K = exp(Lx) exp(Ly)^T in the log domain, FP64.

    The appendix's listing is garbled (its interpolation mixes zeta with itself,
    the function it differentiates is unnamed, the untouched block is assigned an
    undefined iterate, L is halved twice); this follows the accelerated
    alternating minimisation it cites (Guminov et al. 2019), restated:
    minimise phi (``dual_phi``) from eta = zeta = 0, A = 0, with an estimate L of
    the gradient's Lipschitz constant, halved at the start of every iteration and
    doubled after every rejected attempt.  One attempt:
        a_+  = 1/(2L) + sqrt(1/(4L^2) + A/L)      (the root of L a^2 = A + a)
        tau  = a_+ / (A + a_+)
        lam  = tau zeta + (1 - tau) eta
        g    = grad phi(lam) = (P 1 - a, P^T 1 - b),  P = diag(e^lam1) K diag(e^lam2) / c
        eta' = lam with the block of larger ||g_i|| replaced by its exact minimiser,
               a Sinkhorn half-step: eta1' = log a - log K e^lam2 (block 1) or
               eta2' = log b - log K^T e^lam1 (block 2)
        accept when phi(eta') <= phi(lam) - ||g||^2 / (2 L).
    After an accepted attempt zeta <- zeta - a_+ g, eta <- eta', A <- A + a_+.
    An iteration that needs more than ``MAX_ATTEMPTS`` attempts ends the run: the
    required decrease has fallen below what the arithmetic resolves, i.e. eta is
    stationary to working precision (``stopped`` is then set and fewer than
    ``iters`` iterations are reported).
    The averaged primal plan of the listing (n x m) is not formed.

    Returns log u = eta1, log v = eta2 after ``iters`` accepted iterations, the
    value phi(eta) after each, A_k, L_k, the attempts of each iteration, the
    blocks chosen, the smallest relative margins of the two decisions (block
    choice over the attempts without an exact tie, acceptance), the number of
    exact ties (block 1 is taken), the largest |entry| of zeta and eta over
    the run, and ||P 1 - a||_1 + ||P^T 1 - b||_1 at the final eta.
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    loga, logb = np.log(a), np.log(b)
    eta1, eta2 = np.zeros(Lx.shape[0]), np.zeros(Ly.shape[0])
    zeta1, zeta2 = eta1.copy(), eta2.copy()
    A, L = 0.0, float(L0)
    phis, As, Ls, attempts, blocks = [], [], [], [], []
    block_margin, accept_margin = np.inf, np.inf
    ties = 0
    vmax = 0.0  # largest |entry| of zeta and eta over the run
    stopped = False
    for _ in range(iters):
        L_prev = L
        L = L / 2.0
        tries = 0
        accepted = False
        while tries < MAX_ATTEMPTS:
            tries += 1
            an = 1.0 / (2.0 * L) + math.sqrt(1.0 / (4.0 * L * L) + A / L)
            tau = an / (A + an)
            lam1 = tau * zeta1 + (1.0 - tau) * eta1
            lam2 = tau * zeta2 + (1.0 - tau) * eta2
            logKv, _ = _log_Kv(Lx, Ly, lam2)       # log K e^lam2
            logKtu, _ = _log_Kv(Ly, Lx, lam1)      # log K^T e^lam1
            logc = float(lse(lam1 + logKv, axis=0))
            g1 = np.exp(lam1 + logKv - logc) - a
            g2 = np.exp(lam2 + logKtu - logc) - b
            n1, n2 = float(g1 @ g1), float(g2 @ g2)
            phi_lam = logc - lam1 @ a - lam2 @ b
            blk = 1 if n1 >= n2 else 2
            if blk == 1:
                new1, new2 = loga - logKv, lam2
            else:
                new1, new2 = lam1, logb - logKtu
            phi_new = dual_phi(Lx, Ly, a, b, new1, new2)
            bound = phi_lam - (n1 + n2) / (2.0 * L)
            if n1 == n2:
                ties += 1  # exact: blocks holding the same data (self terms of Eq. (2))
            elif n1 + n2 > 0:
                block_margin = min(block_margin, abs(n1 - n2) / (n1 + n2))
            accept_margin = min(accept_margin, abs(phi_new - bound) / max(1.0, abs(bound)))
            if phi_new <= bound:
                accepted = True
                break
            L = 2.0 * L
        if not accepted:
            stopped = True
            L = L_prev
            break
        zeta1, zeta2 = zeta1 - an * g1, zeta2 - an * g2
        eta1, eta2 = new1, new2
        vmax = max(vmax, float(np.abs(zeta1).max()), float(np.abs(zeta2).max()),
                   float(np.abs(eta1).max()), float(np.abs(eta2).max()))
        A += an
        phis.append(phi_new)
        As.append(A)
        Ls.append(L)
        attempts.append(tries)
        blocks.append(blk)
    logKv, _ = _log_Kv(Lx, Ly, eta2)
    logKtu, _ = _log_Kv(Ly, Lx, eta1)
    logc = float(lse(eta1 + logKv, axis=0))
    residual = float(np.abs(np.exp(eta1 + logKv - logc) - a).sum()
                     + np.abs(np.exp(eta2 + logKtu - logc) - b).sum())
    return {"logu": eta1, "logv": eta2, "phi": phis, "A": As, "L": Ls, "attempts": attempts,
            "blocks": blocks, "block_margin": block_margin, "accept_margin": accept_margin,
            "residual": residual, "iters": len(phis), "stopped": stopped, "ties": ties,
            "vmax": vmax}


def sinkhorn_dense(K: np.ndarray, a: np.ndarray, b: np.ndarray, iters: int) -> dict:
    """Textbook Alg. 1 on an explicit positive matrix K (tiny n only), FP64."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    v = np.ones(K.shape[1])
    u = np.ones(K.shape[0])
    for _ in range(iters):
        u = a / (K @ v)
        v = b / (K.T @ u)
    residual = float(np.abs(u * (K @ v) - a).sum())
    return {"u": u, "v": v, "logu": np.log(u), "logv": np.log(v), "residual": residual}


def dual_estimate(a, b, logu, logv, eps: float) -> float:
    """Eq. (6): W_hat = eps (a^T log u + b^T log v)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(eps * (a @ logu + b @ logv))


def dual_objective(a, b, logu, logv, logK: np.ndarray, eps: float) -> float:
    """Eq. (5) objective at alpha = eps log u, beta = eps log v (dense K, tiny n)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    mass = np.exp(logu[:, None] + logK + logv[None, :]).sum()
    return float(eps * (a @ logu) + eps * (b @ logv) - eps * mass + eps)


def primal_objective(logu, logv, logK: np.ndarray, eps: float) -> float:
    """Eq. (3) objective <P, C> - eps H(P) + eps at P = diag(u) K diag(v).

    C = -eps log K (Eq. 7 with K = K_theta) and H(P) = -sum P (log P - 1).
    """
    logP = logu[:, None] + logK + logv[None, :]
    P = np.exp(logP)
    C = -eps * logK
    H = -(P * (logP - 1.0)).sum()
    return float((P * C).sum() - eps * H + eps)


# --------------------------------------------------------------------------
# Full path: theta, W, debiased W_bar
# --------------------------------------------------------------------------

class Theta:
    """Frozen feature parameters theta = (q, U) shared by all terms of Eq. (2)."""

    def __init__(self, q: float, sigma: float, U: np.ndarray, eps: float, R: float):
        self.q, self.sigma, self.U, self.eps, self.R = q, sigma, U, eps, R


def make_theta(X, Y, Z, eps: float) -> Theta:
    """R from both clouds, (q, sigma) from Lemma 1, anchors U = sigma Z."""
    R = radius(X, Y)
    d = np.asarray(X).shape[1]
    q, sigma = gaussian_params(R, eps, d)
    return Theta(q, sigma, anchors(Z, sigma), eps, R)


def solve(Lx, Ly, a, b, iters, mode="log"):
    if mode == "log":
        return sinkhorn_log(Lx, Ly, a, b, iters)
    if mode == "scaled":
        return sinkhorn_scaled(Lx, Ly, a, b, iters)
    raise ValueError(mode)


def divergence(X, Y, a, b, Z=None, eps=None, iters=100, theta: Theta | None = None,
               debiased: bool = True, mode: str = "log") -> dict:
    """W(a,b) and, if asked, W(a,a), W(b,b) and W_bar (Eq. 2) with one theta.

    theta is computed from (X, Y, Z, eps) unless given (it is given, frozen,
    when differentiating).
    """
    if theta is None:
        theta = make_theta(X, Y, Z, eps)
    eps = theta.eps
    Lx = log_features(X, theta.U, eps, theta.q)
    Ly = log_features(Y, theta.U, eps, theta.q)
    out = {"theta": theta}
    sxy = solve(Lx, Ly, a, b, iters, mode)
    out["xy"] = sxy
    out["W_xy"] = dual_estimate(a, b, sxy["logu"], sxy["logv"], eps)
    out["res_xy"] = sxy["residual"]
    if debiased:
        sxx = solve(Lx, Lx, a, a, iters, mode)
        syy = solve(Ly, Ly, b, b, iters, mode)
        out["xx"], out["yy"] = sxx, syy
        out["W_xx"] = dual_estimate(a, a, sxx["logu"], sxx["logv"], eps)
        out["W_yy"] = dual_estimate(b, b, syy["logu"], syy["logv"], eps)
        out["res_xx"], out["res_yy"] = sxx["residual"], syy["residual"]
        out["W_bar"] = out["W_xy"] - 0.5 * (out["W_xx"] + out["W_yy"])
    return out


def divergence_tol(X, Y, a, b, Z, eps, max_iters, tol, check_every=1,
                   debiased: bool = True) -> dict:
    """``divergence`` with Alg. 1's stopping rule on each term of Eq. (2): every
    term runs ``sinkhorn_log_tol`` on its own (its own iteration count)."""
    theta = make_theta(X, Y, Z, eps)
    Lx = log_features(X, theta.U, eps, theta.q)
    Ly = log_features(Y, theta.U, eps, theta.q)
    out = {"theta": theta}
    terms = [("xy", Lx, Ly, a, b)]
    if debiased:
        terms += [("xx", Lx, Lx, a, a), ("yy", Ly, Ly, b, b)]
    for name, L1, L2, w1, w2 in terms:
        st = sinkhorn_log_tol(L1, L2, w1, w2, max_iters, tol, check_every)
        out[name] = st
        out["W_" + name] = dual_estimate(w1, w2, st["logu"], st["logv"], eps)
        out["res_" + name] = st["residual"]
        out["iters_" + name] = st["iters"]
    if debiased:
        out["W_bar"] = out["W_xy"] - 0.5 * (out["W_xx"] + out["W_yy"])
    return out


# --------------------------------------------------------------------------
# Envelope gradient (Prop. 3.3 and the chain rule of Sec. 3.3)
# --------------------------------------------------------------------------

def _grad_points(P, U, L, logu, lt):
    """sum_k exp(log u_i + L_ik + lt_k) * 4 (p_i - u_k), for every row p_i.

    This is -eps sum_k u_i (zeta^T v)_k d xi_ik / d p_i with
    d xi_ik / d p_i = xi_ik * (-4/eps)(p_i - u_k).
    """
    Mass = np.exp(logu[:, None] + L + lt[None, :])
    return 4.0 * (Mass.sum(axis=1)[:, None] * P - Mass @ U)


def gradient(X, Y, a, b, theta: Theta, state: dict, debiased: bool = True) -> dict:
    """Envelope gradient of W (or W_bar) w.r.t. X, Y, a, b, theta held fixed.

    For W(a,b): dW/dK = -eps u v^T (Prop. 3.3), K = xi zeta^T, so
      grad_X = -eps (d xi/dX)^T u (zeta^T v)^T  (formula after Prop. 3.3),
      grad_Y = -eps (d zeta/dY)^T v (xi^T u)^T,
      grad_a = eps log u, grad_b = eps log v  (alpha* = eps log u*, Eq. 5).
    For W(a,a) the kernel is xi xi^T, so X enters both factors:
      dW/dxi = -eps (u (xi^T v)^T + v (xi^T u)^T), grad_a = eps (log u + log v).
    ``state`` is the output of ``divergence``; the potentials are those of its
    final iterate.  Gradients w.r.t. weights are defined up to a constant.
    """
    eps = theta.eps
    U = theta.U
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Lx = log_features(X, U, eps, theta.q)
    Ly = log_features(Y, U, eps, theta.q)
    s = state["xy"]
    lt_v = lse(Ly + s["logv"][:, None], axis=0)     # log zeta^T v
    lt_u = lse(Lx + s["logu"][:, None], axis=0)     # log xi^T u
    gX = _grad_points(X, U, Lx, s["logu"], lt_v)
    gY = _grad_points(Y, U, Ly, s["logv"], lt_u)
    ga = eps * s["logu"]
    gb = eps * s["logv"]
    out = {"W": {"X": gX, "Y": gY, "a": ga, "b": gb}}
    if debiased:
        gx_xx, ga_xx = _grad_self(X, U, Lx, state["xx"], eps)
        gy_yy, gb_yy = _grad_self(Y, U, Ly, state["yy"], eps)
        out["W_bar"] = {"X": gX - 0.5 * gx_xx, "Y": gY - 0.5 * gy_yy,
                        "a": ga - 0.5 * ga_xx, "b": gb - 0.5 * gb_yy}
    return out


def _grad_self(P, U, L, s, eps):
    """Gradient of W(w,w) on one cloud (kernel xi xi^T) w.r.t. its points and weights."""
    lt_v = lse(L + s["logv"][:, None], axis=0)
    lt_u = lse(L + s["logu"][:, None], axis=0)
    g = _grad_points(P, U, L, s["logu"], lt_v) + _grad_points(P, U, L, s["logv"], lt_u)
    return g, eps * (s["logu"] + s["logv"])


def _grad_anchors(P, U, L, logw, lt, q):
    """-sum_i exp(log w_i + L_ik + lt_k) * (4 (p_i - u_k) + 2 u_k / q), for every anchor u_k.

    This is -eps sum_i w_i t_k d xi_ik / d u_k with
    log xi_ik = (d/4) log 2q - (1/2) log r - (2/eps)||p_i - u_k||^2 + ||u_k||^2/(eps q)
    (Lemma 1, proof form), so d xi_ik / d u_k = xi_ik ((4/eps)(p_i - u_k) + 2 u_k/(eps q)).
    """
    Mass = np.exp(logw[:, None] + L + lt[None, :])
    return -4.0 * (Mass.T @ P) + (4.0 - 2.0 / q) * Mass.sum(axis=0)[:, None] * U


def anchor_gradient(X, Y, theta: Theta, state: dict, debiased: bool = True) -> np.ndarray:
    """Envelope gradient of W (or W_bar) w.r.t. the anchors U (r x d), q held fixed.

    Same chain as ``gradient`` (dW/dK = -eps u v^T at the optimum, Prop. 3.3),
    taken through the anchors instead of the points: every feature of both
    clouds depends on u_k, through ||p - u_k||^2 and the weight ||u_k||^2/(eps q).
    For W(a,a) both factors of xi xi^T depend on U.  Learning U (a learned
    feature map, Sec. 3.3) needs exactly this block.
    """
    eps, U, q = theta.eps, theta.U, theta.q
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Lx = log_features(X, U, eps, q)
    Ly = log_features(Y, U, eps, q)
    s = state["xy"]
    lt_v = lse(Ly + s["logv"][:, None], axis=0)
    lt_u = lse(Lx + s["logu"][:, None], axis=0)
    g = _grad_anchors(X, U, Lx, s["logu"], lt_v, q) + _grad_anchors(Y, U, Ly, s["logv"], lt_u, q)
    if debiased:
        for P, L, key in ((X, Lx, "xx"), (Y, Ly, "yy")):
            t = state[key]
            g_self = (_grad_anchors(P, U, L, t["logu"], lse(L + t["logv"][:, None], axis=0), q)
                      + _grad_anchors(P, U, L, t["logv"], lse(L + t["logu"][:, None], axis=0), q))
            g = g - 0.5 * g_self
    return g


# --------------------------------------------------------------------------
# Arc-cosine positive features (Sec. 3.2 "Arc-cosine kernels"; lemma in App. A)
# --------------------------------------------------------------------------

def arccos_kernel(X, Y, s: int) -> np.ndarray:
    """k_s(x, y) = int Theta_s(u.x) Theta_s(u.y) dN(0, I)(u), Theta_s(w) = sqrt(2) max(0, w)^s.

    Closed form for s = 0, 1, 2 (Cho and Saul's arc-cosine kernels, the source the
    paper cites): k_s = ||x||^s ||y||^s J_s(angle) / pi with J_0 = pi - t,
    J_1 = sin t + (pi - t) cos t, J_2 = 3 sin t cos t + (pi - t)(1 + 2 cos^2 t).
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    nx = np.sqrt((X * X).sum(axis=1))
    ny = np.sqrt((Y * Y).sum(axis=1))
    cos = np.clip((X @ Y.T) / (nx[:, None] * ny[None, :]), -1.0, 1.0)
    t = np.arccos(cos)
    if s == 0:
        J = np.pi - t
    elif s == 1:
        J = np.sin(t) + (np.pi - t) * cos
    elif s == 2:
        J = 3.0 * np.sin(t) * cos + (np.pi - t) * (1.0 + 2.0 * cos * cos)
    else:
        raise ValueError("closed form for s = 0, 1, 2 only")
    return (nx[:, None] ** s) * (ny[None, :] ** s) * J / np.pi


def arccos_log_features(P: np.ndarray, U: np.ndarray, s: int, sigma: float,
                        kappa: float) -> np.ndarray:
    """log phi_theta(p) for the perturbed arc-cosine kernel k_s + kappa.

    Per anchor u_k ~ N(0, sigma^2 I) (sigma > 1) the lemma's map has two entries,
    sigma^{d/2} sqrt(2) max(0, u.p)^s exp(-||u||^2 (1 - 1/sigma^2) / 4) and
    sqrt(kappa); phi_theta scales both by r^{-1/2}. The r constant entries only
    ever enter K through their sum kappa, so they are merged into one last
    feature sqrt(kappa): r + 1 features. Entries with u.p <= 0 are 0 (log -inf;
    max(0, w)^0 is taken as 0 for w <= 0). Returns n x (r + 1) in FP64.
    """
    P = np.asarray(P, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    r, d = U.shape
    unorm2 = (U * U).sum(axis=1)
    const = (0.5 * d) * math.log(sigma) + 0.5 * math.log(2.0) - 0.5 * math.log(r) \
        - 0.25 * unorm2 * (1.0 - 1.0 / sigma ** 2)
    W = P @ U.T
    out = np.full((P.shape[0], r + 1), -np.inf)
    pos = W > 0
    logw = np.log(np.where(pos, W, 1.0))  # only read where u.p > 0
    out[:, :r] = np.where(pos, const[None, :] + s * logw, -np.inf)
    out[:, r] = 0.5 * math.log(kappa)
    return out


def arccos_divergence(X, Y, a, b, U, s: int, sigma: float, kappa: float, eps: float = 1.0,
                      iters: int = 100, debiased: bool = True, mode: str = "log") -> dict:
    """Alg. 1 and Eq. (6)/(2) on K = xi zeta^T with arc-cosine features; eps scales W
    (the kernel has no bandwidth: the cost is -eps log k)."""
    Lx = arccos_log_features(X, U, s, sigma, kappa)
    Ly = arccos_log_features(Y, U, s, sigma, kappa)
    out = {}
    sxy = solve(Lx, Ly, a, b, iters, mode)
    out["xy"] = sxy
    out["W_xy"] = dual_estimate(a, b, sxy["logu"], sxy["logv"], eps)
    out["res_xy"] = sxy["residual"]
    if debiased:
        sxx = solve(Lx, Lx, a, a, iters, mode)
        syy = solve(Ly, Ly, b, b, iters, mode)
        out["W_xx"] = dual_estimate(a, a, sxx["logu"], sxx["logv"], eps)
        out["W_yy"] = dual_estimate(b, b, syy["logu"], syy["logv"], eps)
        out["res_xx"], out["res_yy"] = sxx["residual"], syy["residual"]
        out["W_bar"] = out["W_xy"] - 0.5 * (out["W_xx"] + out["W_yy"])
    return out


def deviation(rot: float, rot_hat: float) -> float:
    """Deviation from ground truth used in Sec. 4: D = 100 (ROT - ROT_hat)/|ROT| + 100."""
    return 100.0 * (rot - rot_hat) / abs(rot) + 100.0
