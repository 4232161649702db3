"""Linear-time Sinkhorn divergences with positive features on GB300 (sm_103a).

Python binding of libsinkhorn_pf.so. The ``lsf_*`` functions mirror the C entry
points of include/sinkhorn_pf.h one to one (argument marshalling only: every
step runs in the CUDA kernels). PyTorch provides device memory and streams.

Above them, :class:`SinkhornProblem` keeps one problem resident on the device
(theta, features, scalings, results, workspace), :func:`sinkhorn_divergence`
runs it once, and :class:`SinkhornDivergenceFn` is the autograd wrapper whose
backward pass calls the adjoint kernels.

Paper: Scetbon & Cuturi, "Linear Time Sinkhorn Divergences using Positive
Features", arXiv 2006.07057 (Lemma 1, Alg. 1, Eqs. (2), (6), Prop. 3.3).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from ._binding import (LSF_ERR_NONFINITE, LSF_ERR_TIMEOUT, LSF_KERNEL_FEATURES,  # noqa: F401
                       LSF_KERNEL_OTHER, LSF_KERNEL_PASS, LSF_KERNEL_PASS_RECOMPUTE,
                       LSF_MODE_RECOMPUTE, LSF_MODE_STORED, RESULT_BYTES, LsfCloud, LsfError,
                       LsfResult, LsfScalings, LsfTheta, check, header_symbols, lib)

MODES = {"stored": LSF_MODE_STORED, "recompute": LSF_MODE_RECOMPUTE}

RESULT_DTYPE = np.dtype([("W", "<f8"), ("residual", "<f8"), ("log_scale", "<f8"),
                         ("status", "<i4"), ("iters", "<i4")])
assert RESULT_DTYPE.itemsize == RESULT_BYTES


# ---------------------------------------------------------------- marshalling

def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f32(t):
    if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return t


def ldr_for(r: int) -> int:
    """Row stride of stored features: r rounded up to a multiple of 4."""
    return (r + 3) // 4 * 4


@dataclass
class Theta:
    """Frozen feature parameters (Lemma 1): anchors U, log-constants c, and R, q, sigma."""

    U: torch.Tensor
    c: torch.Tensor
    r: int
    ldr: int
    d: int
    eps: float
    R: float = 0.0
    q: float = 0.0
    sigma: float = 0.0

    def as_c(self) -> LsfTheta:
        return LsfTheta(_p(self.U), _p(self.c), self.r, self.ldr, self.d, float(self.eps))


@dataclass
class Cloud:
    """One weighted cloud: points X, stored features F (or None), row shifts, weights."""

    X: torch.Tensor | None
    F: torch.Tensor | None
    shift: torch.Tensor
    w: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.shift.shape[0])

    def as_c(self) -> LsfCloud:
        return LsfCloud(_p(self.X), _p(self.F), _p(self.shift), _p(self.w), self.n)


@dataclass
class Scalings:
    """Shifted scalings u~ (n), v~ (m) and the r-vectors t_u = xi~^T u~, t_v = zeta~^T v~."""

    u: torch.Tensor
    v: torch.Tensor
    t_u: torch.Tensor
    t_v: torch.Tensor

    @staticmethod
    def alloc(n: int, m: int, ldr: int, device) -> "Scalings":
        z = lambda k: torch.zeros(k, dtype=torch.float32, device=device)  # noqa: E731
        return Scalings(z(n), z(m), z(ldr), z(ldr))

    def as_c(self) -> LsfScalings:
        return LsfScalings(_p(self.u), _p(self.v), _p(self.t_u), _p(self.t_v))


# ---------------------------------------------------------------- C entry points

def lsf_version() -> int:
    return lib().lsf_version()


def lsf_gaussian_params(R: float, eps: float, d: int) -> tuple[float, float]:
    """Lemma 1: (q, sigma) from R, eps, d (host computation in the library)."""
    q = ctypes.c_double()
    s = ctypes.c_double()
    check(lib().lsf_gaussian_params(float(R), float(eps), int(d), ctypes.byref(q),
                                    ctypes.byref(s)), "lsf_gaussian_params")
    return q.value, s.value


def lsf_radius(X, Y, R_out=None, stream=None):
    _f32(X), _f32(Y)
    if R_out is None:
        R_out = torch.empty(1, dtype=torch.float32, device=X.device)
    check(lib().lsf_radius(_p(X), X.shape[0], _p(Y), Y.shape[0], X.shape[1], _p(R_out),
                           _stream(stream)), "lsf_radius")
    return R_out


def lsf_anchors(Z, q, sigma, eps, U=None, c=None, stream=None):
    _f32(Z)
    r, d = Z.shape
    if U is None:
        U = torch.empty(r, d, dtype=torch.float32, device=Z.device)
    if c is None:
        c = torch.empty(r, dtype=torch.float32, device=Z.device)
    check(lib().lsf_anchors(_p(Z), r, d, float(q), float(sigma), float(eps), _p(U), _p(c),
                            _stream(stream)), "lsf_anchors")
    return U, c


def lsf_features(X, theta: Theta, F=None, shift=None, spread=None, stream=None):
    _f32(X)
    n = X.shape[0]
    if F is None:
        F = torch.empty(n, theta.ldr, dtype=torch.float32, device=X.device)
    if shift is None:
        shift = torch.empty(n, dtype=torch.float32, device=X.device)
    th = theta.as_c()
    check(lib().lsf_features(_p(X), n, ctypes.byref(th), _p(F), _p(shift), _p(spread),
                             _stream(stream)), "lsf_features")
    return F, shift


def lsf_row_shift(X, theta: Theta, shift=None, spread=None, stream=None):
    _f32(X)
    n = X.shape[0]
    if shift is None:
        shift = torch.empty(n, dtype=torch.float32, device=X.device)
    th = theta.as_c()
    check(lib().lsf_row_shift(_p(X), n, ctypes.byref(th), _p(shift), _p(spread),
                              _stream(stream)), "lsf_row_shift")
    return shift


def lsf_workspace_bytes(ldr: int) -> int:
    b = ctypes.c_size_t()
    check(lib().lsf_workspace_bytes(int(ldr), ctypes.byref(b)), "lsf_workspace_bytes")
    return b.value


def alloc_workspace(ldr: int, device) -> torch.Tensor:
    nbytes = lsf_workspace_bytes(ldr)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-ws.data_ptr()) % 256
    return ws[off:off + nbytes]


def alloc_results(k: int, device) -> torch.Tensor:
    return torch.zeros(k * RESULT_BYTES, dtype=torch.uint8, device=device)


def lsf_solve(theta: Theta, x: Cloud, y: Cloud, iters: int, mode: str, out: Scalings,
              result, workspace, stream=None):
    th, cx, cy, so = theta.as_c(), x.as_c(), y.as_c(), out.as_c()
    check(lib().lsf_solve(ctypes.byref(th), ctypes.byref(cx), ctypes.byref(cy), int(iters),
                          MODES[mode], ctypes.byref(so), _p(result), _p(workspace),
                          workspace.numel(), _stream(stream)), "lsf_solve")


def lsf_solve_noalloc(theta: Theta, x: Cloud, y: Cloud, iters: int, mode: str, out: Scalings,
                      result, stream=None):
    """lsf_solve without a workspace, for callers that cannot allocate device memory.

    The scratch comes from a fixed 2 MiB array inside the library; calls that can
    overlap on the GPU share it and must not run concurrently.
    """
    th, cx, cy, so = theta.as_c(), x.as_c(), y.as_c(), out.as_c()
    check(lib().lsf_solve_noalloc(ctypes.byref(th), ctypes.byref(cx), ctypes.byref(cy),
                                  int(iters), MODES[mode], ctypes.byref(so), _p(result),
                                  _stream(stream)), "lsf_solve_noalloc")


def lsf_debiased(theta: Theta, x: Cloud, y: Cloud, iters: int, mode: str, s_xy: Scalings,
                 s_xx: Scalings, s_yy: Scalings, result, wbar, workspace, stream=None):
    th, cx, cy = theta.as_c(), x.as_c(), y.as_c()
    a, b, c = s_xy.as_c(), s_xx.as_c(), s_yy.as_c()
    check(lib().lsf_debiased(ctypes.byref(th), ctypes.byref(cx), ctypes.byref(cy), int(iters),
                             MODES[mode], ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                             _p(result), _p(wbar), _p(workspace), workspace.numel(),
                             _stream(stream)), "lsf_debiased")


def lsf_divergence(theta: Theta, xs, ys, ss, results, coef=None, combined=None, workspace=None,
                   stream=None):
    k = len(xs)
    th = theta.as_c()
    cx = [c.as_c() for c in xs]
    cy = [c.as_c() for c in ys]
    cs = [s.as_c() for s in ss]
    PX = (ctypes.POINTER(LsfCloud) * k)(*[ctypes.pointer(c) for c in cx])
    PY = (ctypes.POINTER(LsfCloud) * k)(*[ctypes.pointer(c) for c in cy])
    PS = (ctypes.POINTER(LsfScalings) * k)(*[ctypes.pointer(c) for c in cs])
    PR = (ctypes.c_void_p * k)(*[r.data_ptr() for r in results])
    co = (ctypes.c_double * k)(*(coef if coef is not None else [1.0] * k))
    check(lib().lsf_divergence(ctypes.byref(th), k, PX, PY, PS, PR, co, _p(combined),
                               _p(workspace), workspace.numel(), _stream(stream)),
          "lsf_divergence")


def lsf_gradient(theta: Theta, x: Cloud, y: Cloud, s_xy: Scalings, s_xx: Scalings | None,
                 s_yy: Scalings | None, result, debiased: bool, gX=None, gY=None, ga=None,
                 gb=None, stream=None):
    th, cx, cy = theta.as_c(), x.as_c(), y.as_c()
    a = s_xy.as_c()
    b = s_xx.as_c() if s_xx is not None else None
    c = s_yy.as_c() if s_yy is not None else None
    check(lib().lsf_gradient(ctypes.byref(th), ctypes.byref(cx), ctypes.byref(cy),
                             ctypes.byref(a), ctypes.byref(b) if b else None,
                             ctypes.byref(c) if c else None, _p(result), int(bool(debiased)),
                             _p(gX), _p(gY), _p(ga), _p(gb), _stream(stream)), "lsf_gradient")


def lsf_set_pass_tiling(tile_bytes: int, max_stages: int) -> None:
    check(lib().lsf_set_pass_tiling(int(tile_bytes), int(max_stages)), "lsf_set_pass_tiling")


def lsf_get_pass_tiling() -> tuple[int, int]:
    tb = ctypes.c_int()
    st = ctypes.c_int()
    check(lib().lsf_get_pass_tiling(ctypes.byref(tb), ctypes.byref(st)), "lsf_get_pass_tiling")
    return tb.value, st.value


def lsf_profile_enable(on: bool) -> None:
    check(lib().lsf_profile_enable(int(bool(on))), "lsf_profile_enable")


def lsf_profile_read(kernel_class: int) -> tuple[float, int, float]:
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    by = ctypes.c_double()
    check(lib().lsf_profile_read(int(kernel_class), ctypes.byref(ms), ctypes.byref(n),
                                 ctypes.byref(by)), "lsf_profile_read")
    return ms.value, n.value, by.value


def lsf_launch_count() -> int:
    return int(lib().lsf_launch_count())


def lsf_launch_count_reset() -> None:
    lib().lsf_launch_count_reset()


def read_results(result: torch.Tensor) -> list[dict]:
    """Copy device lsf_result records to the host as dicts."""
    raw = result.cpu().numpy().view(RESULT_DTYPE)
    return [{k: (float(r[k]) if k in ("W", "residual", "log_scale") else int(r[k]))
             for k in RESULT_DTYPE.names} for r in raw]


# ---------------------------------------------------------------- resident problem

class SinkhornProblem:
    """One divergence problem kept resident on the device.

    Builds theta (R from both clouds, q and sigma from Lemma 1, anchors
    U = sigma Z), the row shifts and, in stored mode, the shifted features of
    both clouds; allocates scalings for the three solves of Eq. (2), result
    records and the workspace. ``run`` launches the solve asynchronously;
    ``values`` reads the scalars back.
    """

    def __init__(self, X, Y, a, b, Z, eps: float, mode: str = "stored", ldr: int | None = None,
                 theta: Theta | None = None, stream=None):
        if mode not in MODES:
            raise ValueError(f"mode must be one of {sorted(MODES)}")
        for t in (X, Y, a, b, Z):
            _f32(t)
        self.X, self.Y, self.a, self.b, self.Z = X, Y, a, b, Z
        self.eps = float(eps)
        self.mode = mode
        self.stream = stream
        dev = X.device
        n, d = X.shape
        m = Y.shape[0]
        r = Z.shape[0]
        if theta is None:
            R = float(lsf_radius(X, Y, stream=stream).item())
            q, sigma = lsf_gaussian_params(R, eps, d)
            ldr = ldr if ldr is not None else ldr_for(r)
            U, c = lsf_anchors(Z, q, sigma, eps, stream=stream)
            theta = Theta(U, c, r, ldr, d, self.eps, R, q, sigma)
        self.theta = theta
        ldr = theta.ldr
        self.spread = torch.zeros(1, dtype=torch.float32, device=dev)
        if mode == "stored":
            Fx, sx = lsf_features(X, theta, spread=self.spread, stream=stream)
            Fy, sy = lsf_features(Y, theta, spread=self.spread, stream=stream)
        else:
            Fx = Fy = None
            sx = lsf_row_shift(X, theta, spread=self.spread, stream=stream)
            sy = lsf_row_shift(Y, theta, spread=self.spread, stream=stream)
        self.x = Cloud(X, Fx, sx, a)
        self.y = Cloud(Y, Fy, sy, b)
        self.s_xy = Scalings.alloc(n, m, ldr, dev)
        self.s_xx = Scalings.alloc(n, n, ldr, dev)
        self.s_yy = Scalings.alloc(m, m, ldr, dev)
        self.results = alloc_results(3, dev)
        self.wbar = torch.zeros(1, dtype=torch.float64, device=dev)
        self.workspace = alloc_workspace(ldr, dev)
        self.debiased = None

    def result_view(self, k: int) -> torch.Tensor:
        return self.results[k * RESULT_BYTES:(k + 1) * RESULT_BYTES]

    def run(self, iters: int, debiased: bool = True) -> None:
        """Launch the solve (and Eq. (6)/(2) reductions) on the stream; no host sync."""
        self.debiased = bool(debiased)
        if debiased:
            lsf_debiased(self.theta, self.x, self.y, iters, self.mode, self.s_xy, self.s_xx,
                         self.s_yy, self.results, self.wbar, self.workspace, self.stream)
        else:
            r0 = self.result_view(0)
            lsf_solve(self.theta, self.x, self.y, iters, self.mode, self.s_xy, r0,
                      self.workspace, self.stream)
            lsf_divergence(self.theta, [self.x], [self.y], [self.s_xy], [r0], [1.0], self.wbar,
                           self.workspace, self.stream)

    def values(self) -> dict:
        """Host copy of the results of the last run (synchronises)."""
        recs = read_results(self.results)
        out = {"W_xy": recs[0]["W"], "res_xy": recs[0]["residual"], "status": recs[0]["status"],
               "iters": recs[0]["iters"], "records": recs}
        out["W"] = float(self.wbar.item())
        if self.debiased:
            out.update(W_xx=recs[1]["W"], W_yy=recs[2]["W"], res_xx=recs[1]["residual"],
                       res_yy=recs[2]["residual"], W_bar=out["W"])
        return out

    def gradient(self, debiased: bool | None = None):
        """Envelope gradient of the last run w.r.t. X, Y, a, b (theta fixed)."""
        deb = self.debiased if debiased is None else bool(debiased)
        if deb and not self.debiased:
            raise ValueError("the debiased gradient needs a debiased run")
        dev = self.X.device
        gX = torch.empty_like(self.X)
        gY = torch.empty_like(self.Y)
        ga = torch.empty(self.x.n, dtype=torch.float32, device=dev)
        gb = torch.empty(self.y.n, dtype=torch.float32, device=dev)
        if self.mode != "stored":
            raise NotImplementedError("the adjoint reads stored features")
        lsf_gradient(self.theta, self.x, self.y, self.s_xy, self.s_xx if deb else None,
                     self.s_yy if deb else None, self.results, deb, gX, gY, ga, gb,
                     self.stream)
        return gX, gY, ga, gb


def sinkhorn_divergence(X, Y, a, b, Z, eps: float, iters: int, debiased: bool = True,
                        mode: str = "stored") -> dict:
    """Solve once and return host scalars (W_xy, and W_xx, W_yy, W_bar if debiased)."""
    prob = SinkhornProblem(X, Y, a, b, Z, eps, mode=mode)
    prob.run(iters, debiased=debiased)
    return prob.values()


class SinkhornDivergenceFn(torch.autograd.Function):
    """W (or the debiased W_bar) as a differentiable function of X, Y, a, b.

    theta (R, q, U) is computed from the inputs and then held fixed, as in the
    gradient formula after Prop. 3.3. The backward pass uses the envelope
    gradient of the final iterate; no iteration is replayed.
    """

    @staticmethod
    def forward(ctx, X, Y, a, b, Z, eps, iters, debiased=True):
        prob = SinkhornProblem(X.detach().contiguous(), Y.detach().contiguous(),
                               a.detach().contiguous(), b.detach().contiguous(),
                               Z.detach().contiguous(), eps)
        prob.run(iters, debiased=debiased)
        ctx.prob = prob
        return prob.wbar.to(torch.float32).reshape(())

    @staticmethod
    def backward(ctx, g):
        gX, gY, ga, gb = ctx.prob.gradient()
        return gX * g, gY * g, ga * g, gb * g, None, None, None, None
