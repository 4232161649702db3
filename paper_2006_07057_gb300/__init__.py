"""Linear-time Sinkhorn divergences with positive features on GB300 (sm_103a).

Python binding of libsinkhorn_pf.so. The ``lsf_*`` functions mirror the C entry
points of include/sinkhorn_pf.h one to one (argument marshalling only: every
step runs in the CUDA kernels). PyTorch provides device memory and streams.

Above them, :class:`SinkhornProblem` keeps one problem resident on the device
(theta, features, scalings, results, workspace), :func:`sinkhorn_divergence`
runs it once, and :class:`SinkhornDivergenceFn` is the autograd wrapper whose
backward pass calls the adjoint kernels. :class:`BatchedSolver` runs many
independent problems in one persistent launch, and :class:`MultiSinkhornProblem`
solves many weight pairs on one support with the tensor-core passes.

Paper: Scetbon & Cuturi, "Linear Time Sinkhorn Divergences using Positive
Features", arXiv 2006.07057 (Lemma 1, Alg. 1, Eqs. (2), (6), Prop. 3.3).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from ._binding import (LSF_ERR_ARG, LSF_ERR_UNSUPPORTED, LSF_ERR_WORKSPACE,  # noqa: F401
                       LSF_ERR_NONFINITE, LSF_ERR_TIMEOUT, LSF_KERNEL_ADJOINT,
                       LSF_KERNEL_BATCHED, LSF_KERNEL_SMALL,
                       LSF_KERNEL_FEATURES, LSF_KERNEL_OTHER, LSF_KERNEL_PASS, LSF_KERNEL_PASS_LOG,
                       LsfAccelInfo, LsfBatchInfo, LsfBatchProblem, LsfMultiCloud,
                       LsfMultiScalings, LSF_KERNEL_PASS_MULTI,
                       LSF_KERNEL_PASS_RECOMPUTE, LSF_KERNEL_PASS_HYBRID, LSF_MODE_HYBRID,
                       LSF_MODE_AUTO, LSF_AUTO_SPREAD,
                       LSF_MODE_LOG, LSF_MODE_RECOMPUTE,
                       LSF_MODE_STORED, RESULT_BYTES, LsfCloud, LsfError, LsfResult, LsfScalings,
                       LsfArccos, LsfTheta, LsfPipeline, LsfPipelineOut, LsfPipelineViews, check,
                       header_symbols, lib)

MODES = {"stored": LSF_MODE_STORED, "recompute": LSF_MODE_RECOMPUTE, "log": LSF_MODE_LOG,
         "hybrid": LSF_MODE_HYBRID, "auto": LSF_MODE_AUTO}
MODE_NAMES = {v: k for k, v in MODES.items()}

# The library's "auto" threshold: a problem goes straight to the log domain when
# the within-row log-feature spread exceeds this many nats (the batched solver's
# routing uses the same value).
LOG_SPREAD = LSF_AUTO_SPREAD

RESULT_DTYPE = np.dtype([("W", "<f8"), ("residual", "<f8"), ("log_scale", "<f8"),
                         ("status", "<i4"), ("iters", "<i4"), ("mode", "<i4"), ("reserved", "<i4")])
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
class Arccos:
    """Arc-cosine feature parameters: anchors U = sigma Z, constants c, exponent s, kappa."""

    U: torch.Tensor
    c: torch.Tensor
    r: int
    ldr: int
    d: int
    s: int
    sigma: float
    kappa: float

    def as_c(self) -> LsfArccos:
        return LsfArccos(_p(self.U), _p(self.c), self.r, self.ldr, self.d, int(self.s),
                         float(self.kappa))


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


def lsf_log_features(X, theta: Theta, L=None, shift=None, spread=None, stream=None):
    _f32(X)
    n = X.shape[0]
    if L is None:
        L = torch.empty(n, theta.ldr, dtype=torch.float32, device=X.device)
    if shift is None:
        shift = torch.empty(n, dtype=torch.float32, device=X.device)
    th = theta.as_c()
    check(lib().lsf_log_features(_p(X), n, ctypes.byref(th), _p(L), _p(shift), _p(spread),
                                 _stream(stream)), "lsf_log_features")
    return L, shift


def lsf_row_shift(X, theta: Theta, shift=None, spread=None, stream=None):
    _f32(X)
    n = X.shape[0]
    if shift is None:
        shift = torch.empty(n, dtype=torch.float32, device=X.device)
    th = theta.as_c()
    check(lib().lsf_row_shift(_p(X), n, ctypes.byref(th), _p(shift), _p(spread),
                              _stream(stream)), "lsf_row_shift")
    return shift


def lsf_hybrid_columns(ldr: int) -> int:
    """First stored column c0 of the hybrid pass for row stride ldr."""
    c0 = ctypes.c_int()
    check(lib().lsf_hybrid_columns(int(ldr), ctypes.byref(c0)), "lsf_hybrid_columns")
    return c0.value


def lsf_hybrid_features(X, theta: Theta, Fs=None, shift=None, spread=None, stream=None):
    """Row shifts and the stored block (columns c0..ldr-1) of the hybrid pass."""
    _f32(X)
    n = X.shape[0]
    c0 = lsf_hybrid_columns(theta.ldr)
    if Fs is None:
        Fs = torch.empty(n, theta.ldr - c0, dtype=torch.float32, device=X.device)
    if shift is None:
        shift = torch.empty(n, dtype=torch.float32, device=X.device)
    th = theta.as_c()
    check(lib().lsf_hybrid_features(_p(X), n, ctypes.byref(th), _p(Fs), _p(shift), _p(spread),
                                    _stream(stream)), "lsf_hybrid_features")
    return Fs, shift


def lsf_arccos_anchors(Z, sigma: float, U=None, c=None, stream=None):
    _f32(Z)
    r, d = Z.shape
    if U is None:
        U = torch.empty(r, d, dtype=torch.float32, device=Z.device)
    if c is None:
        c = torch.empty(r, dtype=torch.float32, device=Z.device)
    check(lib().lsf_arccos_anchors(_p(Z), r, d, float(sigma), _p(U), _p(c), _stream(stream)),
          "lsf_arccos_anchors")
    return U, c


def lsf_arccos_features(X, params: Arccos, F=None, shift=None, spread=None, stream=None):
    _f32(X)
    n = X.shape[0]
    if F is None:
        F = torch.empty(n, params.ldr, dtype=torch.float32, device=X.device)
    if shift is None:
        shift = torch.empty(n, dtype=torch.float32, device=X.device)
    pa = params.as_c()
    check(lib().lsf_arccos_features(_p(X), n, ctypes.byref(pa), _p(F), _p(shift), _p(spread),
                                    _stream(stream)), "lsf_arccos_features")
    return F, shift


def lsf_arccos_log_features(X, params: Arccos, L=None, shift=None, spread=None, stream=None):
    _f32(X)
    n = X.shape[0]
    if L is None:
        L = torch.empty(n, params.ldr, dtype=torch.float32, device=X.device)
    if shift is None:
        shift = torch.empty(n, dtype=torch.float32, device=X.device)
    pa = params.as_c()
    check(lib().lsf_arccos_log_features(_p(X), n, ctypes.byref(pa), _p(L), _p(shift), _p(spread),
                                        _stream(stream)), "lsf_arccos_log_features")
    return L, shift


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


def lsf_accel_workspace_bytes(n: int, m: int, ldr: int) -> int:
    b = ctypes.c_size_t(0)
    check(lib().lsf_accel_workspace_bytes(int(n), int(m), int(ldr), ctypes.byref(b)),
          "lsf_accel_workspace_bytes")
    return int(b.value)


def alloc_accel_workspace(n: int, m: int, ldr: int, device) -> torch.Tensor:
    nbytes = lsf_accel_workspace_bytes(n, m, ldr)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-ws.data_ptr()) % 256
    return ws[off:off + nbytes]


def lsf_solve_accelerated(theta: Theta, x: Cloud, y: Cloud, iters: int, out: Scalings, result,
                          workspace, L0: float = 1.0, stream=None) -> dict:
    """Accelerated Sinkhorn (App. A.2) in the log domain; returns the line-search
    statistics (iters, attempts, A, L). Synchronises the stream once per attempt."""
    th, cx, cy, so = theta.as_c(), x.as_c(), y.as_c(), out.as_c()
    info = LsfAccelInfo()
    check(lib().lsf_solve_accelerated(ctypes.byref(th), ctypes.byref(cx), ctypes.byref(cy),
                                      int(iters), float(L0), ctypes.byref(so), _p(result),
                                      ctypes.byref(info), _p(workspace), workspace.numel(),
                                      _stream(stream)), "lsf_solve_accelerated")
    return {"iters": info.iters, "attempts": info.attempts, "A": info.A, "L": info.L}


def lsf_solve_noalloc(theta: Theta, x: Cloud, y: Cloud, iters: int, mode: str, out: Scalings,
                      result, stream=None):
    """lsf_solve without a workspace, for callers that cannot allocate device memory.

    The scratch comes from a fixed 12 MiB array inside the library; calls that can
    overlap on the GPU share it and must not run concurrently.
    """
    th, cx, cy, so = theta.as_c(), x.as_c(), y.as_c(), out.as_c()
    check(lib().lsf_solve_noalloc(ctypes.byref(th), ctypes.byref(cx), ctypes.byref(cy),
                                  int(iters), MODES[mode], ctypes.byref(so), _p(result),
                                  _stream(stream)), "lsf_solve_noalloc")


def pipeline_desc(n: int, m: int, d: int, r: int, eps: float, iters: int, debiased: bool = True,
                  mode: str = "stored", ldr: int = 0) -> LsfPipeline:
    return LsfPipeline(int(n), int(m), int(d), int(r), int(ldr), float(eps), int(iters),
                       int(bool(debiased)), MODES[mode])


def lsf_pipeline_bytes(desc: LsfPipeline) -> int:
    b = ctypes.c_size_t()
    check(lib().lsf_pipeline_bytes(ctypes.byref(desc), ctypes.byref(b)), "lsf_pipeline_bytes")
    return b.value


def lsf_pipeline_run(desc: LsfPipeline, X, Y, a, b, Z, arena, out_ptr: int, stream=None) -> None:
    """Queue the whole path for host arrays X, Y, a, b, Z (contiguous float32 CPU
    tensors, pinned for an asynchronous call) into the device arena; the host
    record lands at out_ptr (sizeof(LsfPipelineOut) bytes, pinned) when the
    stream reaches the end of the call."""
    for t in (X, Y, a, b, Z):
        if t.dtype != torch.float32 or t.is_cuda or not t.is_contiguous():
            raise ValueError("expected contiguous float32 host tensors")
    check(lib().lsf_pipeline_run(ctypes.byref(desc), _p(X), _p(Y), _p(a), _p(b), _p(Z), _p(arena),
                                 arena.numel(), ctypes.cast(ctypes.c_void_p(out_ptr),
                                                            ctypes.POINTER(LsfPipelineOut)),
                                 _stream(stream)), "lsf_pipeline_run")


def lsf_pipeline_layout(desc: LsfPipeline, arena) -> LsfPipelineViews:
    """Device views (theta, clouds, scalings, result records) into a pipeline arena."""
    v = LsfPipelineViews()
    check(lib().lsf_pipeline_layout(ctypes.byref(desc), _p(arena), ctypes.byref(v)),
          "lsf_pipeline_layout")
    return v


def lsf_pipeline_finish(desc: LsfPipeline, arena, out_ptr: int, stream=None) -> None:
    """Eq. (2) from the arena's result records and the host record copy (on the stream)."""
    check(lib().lsf_pipeline_finish(ctypes.byref(desc), _p(arena),
                                    ctypes.cast(ctypes.c_void_p(out_ptr), ctypes.POINTER(LsfPipelineOut)),
                                    _stream(stream)), "lsf_pipeline_finish")


def alloc_arena(nbytes: int, device) -> torch.Tensor:
    """A 256-byte aligned device byte buffer of nbytes."""
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + nbytes]


class HostPipeline:
    """The whole path for problems held in host memory, through lsf_pipeline_run.

    Owns one device arena (grown when a larger problem comes) and a pinned host
    record; ``run`` queues a problem on the stream (no host wait, except in
    ``auto`` mode) and ``result`` waits for it and returns the host values.
    """

    def __init__(self, device=None, stream=None):
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream
        self.arena = None
        self._out = torch.zeros(ctypes.sizeof(LsfPipelineOut), dtype=torch.uint8).pin_memory()
        self.event = torch.cuda.Event()

    def run(self, X, Y, a, b, Z, eps: float, iters: int, debiased: bool = True,
            mode: str = "stored") -> None:
        n, d = X.shape
        desc = pipeline_desc(n, Y.shape[0], d, Z.shape[0], eps, iters, debiased, mode)
        need = lsf_pipeline_bytes(desc)
        if self.arena is None or self.arena.numel() < need:
            self.arena = alloc_arena(need, self.device)
        lsf_pipeline_run(desc, X, Y, a, b, Z, self.arena, self._out.data_ptr(), self.stream)
        self.event.record(self.stream if self.stream is not None else torch.cuda.current_stream())

    def done(self) -> bool:
        return self.event.query()

    def result(self) -> dict:
        self.event.synchronize()
        o = LsfPipelineOut.from_address(self._out.data_ptr())
        return {k: getattr(o, k) for k, _ in LsfPipelineOut._fields_ if k != "reserved"} | {
            "mode_name": MODE_NAMES.get(o.mode, "?")}


def ldr2_for(r: int) -> int:
    """Row stride of the bf16 pair features of the tensor-core pass: r rounded up to 128."""
    return (r + 127) // 128 * 128


def multi_kp(k: int) -> int:
    """Right-hand sides the tensor-core pass computes for k solves (16 or 32)."""
    return 16 if k <= 16 else 32


def lsf_split_features(F: torch.Tensor, r: int, ldr2: int | None = None, F2=None,
                       stream=None) -> torch.Tensor:
    """bf16 pair planes (2 x n x ldr2, hi and lo) of stored FP32 features F (n x ldr)."""
    _f32(F)
    n, ldr = F.shape
    ldr2 = ldr2 if ldr2 is not None else ldr2_for(r)
    if F2 is None:
        F2 = torch.empty((2, n, ldr2), dtype=torch.bfloat16, device=F.device)
    check(lib().lsf_split_features(_p(F), int(n), int(ldr), int(r), _p(F2), int(ldr2),
                                   _stream(stream)), "lsf_split_features")
    return F2


def lsf_set_multi_tuning(prefetch_chunks: int = 0, l2_hints: int = 1,
                         r_vectors_resident: int = 0) -> None:
    """Tuning of the multi-right-hand-side pass: row chunks requested into L2 ahead
    of its ring, the L2 eviction hints of its two reads of each chunk (0, 1, 2),
    and whether the split r-vectors stay in shared memory for the launch."""
    check(lib().lsf_set_multi_tuning(int(prefetch_chunks), int(l2_hints), int(r_vectors_resident)),
          "lsf_set_multi_tuning")


def lsf_multi_workspace_bytes(ldr2: int, k: int) -> int:
    b = ctypes.c_size_t(0)
    check(lib().lsf_multi_workspace_bytes(int(ldr2), int(k), ctypes.byref(b)),
          "lsf_multi_workspace_bytes")
    return int(b.value)


def lsf_solve_multi(theta: Theta, ldr2: int, F2x, shift_x, Wx, F2y, shift_y, Wy, iters: int,
                    U, V, Tu, Tv, results, workspace, stream=None) -> None:
    """Alg. 1 and Eq. (6) for the k weight pairs (rows of Wx, Wy) on one support."""
    k = int(Wx.shape[0])
    th = theta.as_c()
    cx = LsfMultiCloud(_p(F2x), _p(shift_x), _p(Wx), int(Wx.shape[1]))
    cy = LsfMultiCloud(_p(F2y), _p(shift_y), _p(Wy), int(Wy.shape[1]))
    so = LsfMultiScalings(_p(U), _p(V), _p(Tu), _p(Tv))
    check(lib().lsf_solve_multi(ctypes.byref(th), int(ldr2), ctypes.byref(cx), ctypes.byref(cy), k,
                                int(iters), ctypes.byref(so), _p(results), _p(workspace),
                                workspace.numel(), _stream(stream)), "lsf_solve_multi")


def lsf_multi_debiased(theta: Theta, ldr2: int, F2x, shift_x, Wx, F2y, shift_y, Wy, iters: int,
                       s_xy: dict, s_xx: dict, s_yy: dict, results, wbar, workspace,
                       stream=None) -> None:
    """Eq. (2) for the k weight pairs: three multi-pair solves and the per-pair
    combination on the device (results: 3k records xy, xx, yy; wbar: k doubles)."""
    k = int(Wx.shape[0])
    th = theta.as_c()
    cx = LsfMultiCloud(_p(F2x), _p(shift_x), _p(Wx), int(Wx.shape[1]))
    cy = LsfMultiCloud(_p(F2y), _p(shift_y), _p(Wy), int(Wy.shape[1]))
    sc = [LsfMultiScalings(_p(s["U"]), _p(s["V"]), _p(s["Tu"]), _p(s["Tv"]))
          for s in (s_xy, s_xx, s_yy)]
    check(lib().lsf_multi_debiased(ctypes.byref(th), int(ldr2), ctypes.byref(cx), ctypes.byref(cy),
                                   k, int(iters), ctypes.byref(sc[0]), ctypes.byref(sc[1]),
                                   ctypes.byref(sc[2]), _p(results), _p(wbar), _p(workspace),
                                   workspace.numel(), _stream(stream)), "lsf_multi_debiased")


def lsf_debiased(theta: Theta, x: Cloud, y: Cloud, iters: int, mode: str, s_xy: Scalings,
                 s_xx: Scalings, s_yy: Scalings, result, wbar, workspace, stream=None):
    th, cx, cy = theta.as_c(), x.as_c(), y.as_c()
    a, b, c = s_xy.as_c(), s_xx.as_c(), s_yy.as_c()
    check(lib().lsf_debiased(ctypes.byref(th), ctypes.byref(cx), ctypes.byref(cy), int(iters),
                             MODES[mode], ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                             _p(result), _p(wbar), _p(workspace), workspace.numel(),
                             _stream(stream)), "lsf_debiased")


def lsf_solve_tol(theta: Theta, x: Cloud, y: Cloud, max_iters: int, tol: float, check_every: int,
                  mode: str, out: Scalings, result, workspace, stream=None):
    """Alg. 1 until the residual is at most tol (checked every check_every
    iterations); synchronises the stream at every check."""
    th, cx, cy, so = theta.as_c(), x.as_c(), y.as_c(), out.as_c()
    check(lib().lsf_solve_tol(ctypes.byref(th), ctypes.byref(cx), ctypes.byref(cy), int(max_iters),
                              float(tol), int(check_every), MODES[mode], ctypes.byref(so),
                              _p(result), _p(workspace), workspace.numel(), _stream(stream)),
          "lsf_solve_tol")


def lsf_debiased_tol(theta: Theta, x: Cloud, y: Cloud, max_iters: int, tol: float, check_every: int,
                     mode: str, s_xy: Scalings, s_xx: Scalings, s_yy: Scalings, result, wbar,
                     workspace, stream=None):
    """Eq. (2) with each term stopped by Alg. 1's rule; synchronises at every check."""
    th, cx, cy = theta.as_c(), x.as_c(), y.as_c()
    a, b, c = s_xy.as_c(), s_xx.as_c(), s_yy.as_c()
    check(lib().lsf_debiased_tol(ctypes.byref(th), ctypes.byref(cx), ctypes.byref(cy),
                                 int(max_iters), float(tol), int(check_every), MODES[mode],
                                 ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), _p(result),
                                 _p(wbar), _p(workspace), workspace.numel(), _stream(stream)),
          "lsf_debiased_tol")


def lsf_divergence(theta: Theta, xs, ys, ss, results, coef=None, combined=None, workspace=None,
                   stream=None, mode: str = "stored"):
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
                               MODES[mode], _p(workspace), workspace.numel(), _stream(stream)),
          "lsf_divergence")


def lsf_gradient(theta: Theta, x: Cloud, y: Cloud, s_xy: Scalings, s_xx: Scalings | None,
                 s_yy: Scalings | None, result, debiased: bool, gX=None, gY=None, ga=None,
                 gb=None, stream=None, mode: str = "stored"):
    th, cx, cy = theta.as_c(), x.as_c(), y.as_c()
    a = s_xy.as_c()
    b = s_xx.as_c() if s_xx is not None else None
    c = s_yy.as_c() if s_yy is not None else None
    check(lib().lsf_gradient(ctypes.byref(th), ctypes.byref(cx), ctypes.byref(cy),
                             ctypes.byref(a), ctypes.byref(b) if b else None,
                             ctypes.byref(c) if c else None, _p(result), int(bool(debiased)),
                             MODES[mode], _p(gX), _p(gY), _p(ga), _p(gb), _stream(stream)),
          "lsf_gradient")


def lsf_anchor_gradient(theta: Theta, x: Cloud, y: Cloud, s_xy: Scalings, s_xx: Scalings | None,
                        s_yy: Scalings | None, debiased: bool, gU, workspace, scale: float = 1.0,
                        stream=None, mode: str = "stored"):
    th, cx, cy = theta.as_c(), x.as_c(), y.as_c()
    a = s_xy.as_c()
    b = s_xx.as_c() if s_xx is not None else None
    c = s_yy.as_c() if s_yy is not None else None
    check(lib().lsf_anchor_gradient(ctypes.byref(th), float(theta.q), ctypes.byref(cx),
                                    ctypes.byref(cy), ctypes.byref(a),
                                    ctypes.byref(b) if b else None, ctypes.byref(c) if c else None,
                                    int(bool(debiased)), MODES[mode], float(scale), _p(gU),
                                    _p(workspace), workspace.numel(), _stream(stream)),
          "lsf_anchor_gradient")


def lsf_set_batch_strategy(strategy: int) -> None:
    """0: persistent kernel (default), 1: one cluster per problem, 2: by rule."""
    check(lib().lsf_set_batch_strategy(int(strategy)), "lsf_set_batch_strategy")


def lsf_set_batch_fault(wait_limit_ns: int = 4_000_000_000, stall_rounds: int = 0) -> None:
    """Failure-detection hook of the batched solver (tests): the limit of its
    bounded waits, and whether its round flags are made unreachable."""
    check(lib().lsf_set_batch_fault(int(wait_limit_ns), int(stall_rounds)), "lsf_set_batch_fault")


def lsf_set_small_solver(policy: int, max_entries: int = 1 << 24) -> None:
    """0: never use the cluster small-problem solver, 1: by size (default), 2: always."""
    check(lib().lsf_set_small_solver(int(policy), int(max_entries)), "lsf_set_small_solver")


def lsf_set_pass_tiling(tile_bytes: int, max_stages: int) -> None:
    check(lib().lsf_set_pass_tiling(int(tile_bytes), int(max_stages)), "lsf_set_pass_tiling")


def lsf_get_pass_tiling() -> tuple[int, int]:
    tb = ctypes.c_int()
    st = ctypes.c_int()
    check(lib().lsf_get_pass_tiling(ctypes.byref(tb), ctypes.byref(st)), "lsf_get_pass_tiling")
    return tb.value, st.value


def lsf_profile_enable(on: bool) -> None:
    check(lib().lsf_profile_enable(int(bool(on))), "lsf_profile_enable")


def lsf_set_tracing(level: int) -> int:
    """NVTX ranges for a profiler: 0 none, 1 entry points (default), 2 also every
    kernel launch by class. Returns the previous level."""
    prev = ctypes.c_int()
    check(lib().lsf_set_tracing(int(level), ctypes.byref(prev)), "lsf_set_tracing")
    return prev.value


def lsf_profile_read(kernel_class: int) -> tuple[float, int, float]:
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    by = ctypes.c_double()
    check(lib().lsf_profile_read(int(kernel_class), ctypes.byref(ms), ctypes.byref(n),
                                 ctypes.byref(by)), "lsf_profile_read")
    return ms.value, n.value, by.value


def lsf_probe_pipe_rates(stream=None) -> dict:
    """Measured results per clock per SM: packed and scalar FP32 FMA lane operations
    and ex2 (the recompute and hybrid passes' ALU roofline). Synchronises."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(lib().lsf_probe_pipe_rates(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                     _stream(stream)), "lsf_probe_pipe_rates")
    return {"ffma2_lane_ops_per_clk_sm": a.value, "ffma_lane_ops_per_clk_sm": b.value,
            "ex2_per_clk_sm": c.value}


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
    U = sigma Z), the row shifts and the stored features of both clouds
    (shifted features for ``mode="stored"``, their logs for ``mode="log"``,
    none for ``mode="recompute"``); allocates scalings for the three solves of
    Eq. (2), result records and the workspace. ``run`` launches the solve
    asynchronously; ``values`` reads the scalars back.

    ``mode="auto"`` hands the choice of domain to the library (LSF_MODE_AUTO):
    at ``run`` it builds the features itself, goes to the log domain when the
    within-row log-feature spread exceeds ``LOG_SPREAD``, else solves in the
    scaling domain and repeats the solve in the log domain if that run reports a
    non-finite scaling. ``used_mode`` then tells which domain produced the result.
    """

    def __init__(self, X, Y, a, b, Z, eps: float, mode: str = "stored", ldr: int | None = None,
                 theta: Theta | None = None, stream=None, scalings: bool = True,
                 kernel: str = "gaussian", s: int = 1, sigma: float = 1.5, kappa: float = 0.1):
        if mode not in MODES:
            raise ValueError(f"mode must be one of {sorted(MODES)}")
        if kernel not in ("gaussian", "arccos"):
            raise ValueError("kernel must be 'gaussian' or 'arccos'")
        if kernel == "arccos" and mode in ("recompute", "hybrid"):
            raise ValueError("the recompute and hybrid modes evaluate the Gaussian map only")
        self.kernel = kernel
        self.arccos = None
        for t in (X, Y, a, b, Z):
            _f32(t)
        self.X, self.Y, self.a, self.b, self.Z = X, Y, a, b, Z
        self.eps = float(eps)
        self.stream = stream
        self.auto = mode == "auto"
        dev = X.device
        n, d = X.shape
        m = Y.shape[0]
        r = Z.shape[0]
        if kernel == "arccos":
            # r anchors give r + 1 features (the merged constant feature sqrt(kappa))
            ldr = ldr if ldr is not None else ldr_for(r + 1)
            U, c = lsf_arccos_anchors(Z, sigma, stream=stream)
            self.arccos = Arccos(U, c, r, ldr, d, s, float(sigma), float(kappa))
            # the solver reads only ldr and eps; no Gaussian kernel may see these anchors
            theta = Theta(None, None, r + 1, ldr, d, self.eps, 0.0, 0.0, float(sigma))
        elif theta is None:
            R = float(lsf_radius(X, Y, stream=stream).item())
            q, sig = lsf_gaussian_params(R, eps, d)
            ldr = ldr if ldr is not None else ldr_for(r)
            U, c = lsf_anchors(Z, q, sig, eps, stream=stream)
            theta = Theta(U, c, r, ldr, d, self.eps, R, q, sig)
        self.theta = theta
        ldr = theta.ldr
        self.spread = torch.zeros(1, dtype=torch.float32, device=dev)
        if self.auto and kernel == "arccos":
            raise ValueError("auto mode builds Gaussian features; pick a mode for arc-cosine")
        self.mode = mode
        self._build_features()
        self.debiased = None
        self.iters = None
        if not scalings:
            return
        self.s_xy = Scalings.alloc(n, m, ldr, dev)
        self.s_xx = Scalings.alloc(n, n, ldr, dev)
        self.s_yy = Scalings.alloc(m, m, ldr, dev)
        self.results = alloc_results(3, dev)
        self.wbar = torch.zeros(1, dtype=torch.float64, device=dev)
        self.workspace = alloc_workspace(ldr, dev)

    def _build_features(self):
        X, Y, th, st = self.X, self.Y, self.theta, self.stream
        if self.mode == "auto":
            # the library builds the features of the domain it picks into these
            e = lambda *s_: torch.empty(s_, dtype=torch.float32, device=X.device)  # noqa: E731
            self.x = Cloud(X, e(X.shape[0], th.ldr), e(X.shape[0]), self.a)
            self.y = Cloud(Y, e(Y.shape[0], th.ldr), e(Y.shape[0]), self.b)
            return
        if self.arccos is not None:
            build = lsf_arccos_features if self.mode == "stored" else lsf_arccos_log_features
            Fx, sx = build(X, self.arccos, spread=self.spread, stream=st)
            Fy, sy = build(Y, self.arccos, spread=self.spread, stream=st)
            self.x = Cloud(X, Fx, sx, self.a)
            self.y = Cloud(Y, Fy, sy, self.b)
            return
        if self.mode == "stored":
            Fx, sx = lsf_features(X, th, spread=self.spread, stream=st)
            Fy, sy = lsf_features(Y, th, spread=self.spread, stream=st)
        elif self.mode == "log":
            Fx, sx = lsf_log_features(X, th, spread=self.spread, stream=st)
            Fy, sy = lsf_log_features(Y, th, spread=self.spread, stream=st)
        elif self.mode == "hybrid":
            Fx, sx = lsf_hybrid_features(X, th, spread=self.spread, stream=st)
            Fy, sy = lsf_hybrid_features(Y, th, spread=self.spread, stream=st)
        else:
            Fx = Fy = None
            sx = lsf_row_shift(X, th, spread=self.spread, stream=st)
            sy = lsf_row_shift(Y, th, spread=self.spread, stream=st)
        self.x = Cloud(X, Fx, sx, self.a)
        self.y = Cloud(Y, Fy, sy, self.b)

    def switch_mode(self, mode: str) -> None:
        """Rebuild the features for another solver mode (same theta)."""
        if mode != self.mode:
            self.mode = mode
            self._build_features()

    def result_view(self, k: int) -> torch.Tensor:
        return self.results[k * RESULT_BYTES:(k + 1) * RESULT_BYTES]

    def run(self, iters: int, debiased: bool = True, tol: float | None = None,
            check_every: int = 10) -> None:
        """Launch the solve (and Eq. (6)/(2) reductions) on the stream.

        No host synchronisation, except in ``auto`` mode, where the library reads
        the spread and the status back to pick the domain (``used_mode``).
        With ``tol``, Alg. 1's stopping rule: each solve ends at the first check
        (every ``check_every`` iterations, ``iters`` at most) where its residual
        is at most ``tol``; each check reads the residual on the host, and the
        iterations run are in each result record (``values()["iters_*"]``).
        """
        self.debiased = bool(debiased)
        self.iters = iters
        self._used = None
        if tol is None:
            self._launch(iters)
            return
        if self.debiased:
            lsf_debiased_tol(self.theta, self.x, self.y, iters, tol, check_every, self.mode,
                             self.s_xy, self.s_xx, self.s_yy, self.results, self.wbar,
                             self.workspace, self.stream)
        else:
            r0 = self.result_view(0)
            lsf_solve_tol(self.theta, self.x, self.y, iters, tol, check_every, self.mode, self.s_xy,
                          r0, self.workspace, self.stream)
            lsf_divergence(self.theta, [self.x], [self.y], [self.s_xy], [r0], [1.0], self.wbar,
                           self.workspace, self.stream, mode=self.used_mode)

    @property
    def used_mode(self) -> str:
        """The mode the last run's features, scalings and W are in (reads the
        result record once in ``auto`` mode)."""
        if not self.auto:
            return self.mode
        if getattr(self, "_used", None) is None:
            self._used = MODE_NAMES[read_results(self.result_view(0))[0]["mode"]]
        return self._used

    def _launch(self, iters: int) -> None:
        if self.debiased:
            lsf_debiased(self.theta, self.x, self.y, iters, self.mode, self.s_xy, self.s_xx,
                         self.s_yy, self.results, self.wbar, self.workspace, self.stream)
        else:
            r0 = self.result_view(0)
            lsf_solve(self.theta, self.x, self.y, iters, self.mode, self.s_xy, r0,
                      self.workspace, self.stream)
            lsf_divergence(self.theta, [self.x], [self.y], [self.s_xy], [r0], [1.0], self.wbar,
                           self.workspace, self.stream, mode=self.mode)

    def run_accelerated(self, iters: int, debiased: bool = True, L0: float = 1.0) -> list[dict]:
        """Accelerated Sinkhorn (App. A.2) for each solve of the divergence, then Eq. (6)
        (and Eq. (2)). Log domain only (``mode="log"``); synchronises once per
        line-search attempt. Returns the line-search statistics of each solve."""
        if self.mode != "log":
            raise ValueError("the accelerated solver runs in the log domain (mode='log')")
        self.debiased = bool(debiased)
        self.iters = iters
        n, m = self.x.n, self.y.n
        if getattr(self, "_accel_ws", None) is None:
            big = max(n, m)
            self._accel_ws = alloc_accel_workspace(big, big, self.theta.ldr, self.X.device)
        pairs = [(self.x, self.y, self.s_xy)]
        if self.debiased:
            pairs += [(self.x, self.x, self.s_xx), (self.y, self.y, self.s_yy)]
        stats = []
        for k, (cx, cy, s) in enumerate(pairs):
            stats.append(lsf_solve_accelerated(self.theta, cx, cy, iters, s, self.result_view(k),
                                               self._accel_ws, L0=L0, stream=self.stream))
        xs = [p[0] for p in pairs]
        ys = [p[1] for p in pairs]
        coef = [1.0, -0.5, -0.5][:len(pairs)]
        lsf_divergence(self.theta, xs, ys, [p[2] for p in pairs],
                       [self.result_view(k) for k in range(len(pairs))], coef, self.wbar,
                       self.workspace, self.stream, mode="log")
        self.accel_stats = stats
        return stats

    def values(self) -> dict:
        """Host copy of the results of the last run (synchronises)."""
        recs = read_results(self.results)
        out = {"W_xy": recs[0]["W"], "res_xy": recs[0]["residual"], "status": recs[0]["status"],
               "iters": recs[0]["iters"], "iters_xy": recs[0]["iters"], "records": recs,
               "mode": MODE_NAMES[recs[0]["mode"]]}
        out["W"] = float(self.wbar.item())
        if self.debiased:
            out.update(W_xx=recs[1]["W"], W_yy=recs[2]["W"], res_xx=recs[1]["residual"],
                       res_yy=recs[2]["residual"], W_bar=out["W"], iters_xx=recs[1]["iters"],
                       iters_yy=recs[2]["iters"])
        return out

    def log_potentials(self, which: str = "xy"):
        """log u, log v of a solve (undoing the row shifts and the global factor M)."""
        k = {"xy": 0, "xx": 1, "yy": 2}[which]
        s = {"xy": self.s_xy, "xx": self.s_xx, "yy": self.s_yy}[which]
        xs = self.x.shift if which in ("xy", "xx") else self.y.shift
        ys = self.y.shift if which in ("xy", "yy") else self.x.shift
        rec = read_results(self.results)[k]
        M = rec["log_scale"]
        lg = rec["mode"] == LSF_MODE_LOG
        lu = s.u.double() if lg else torch.log(s.u.double())
        lv = s.v.double() if lg else torch.log(s.v.double())
        return lu - xs.double() - M, lv - ys.double() + M

    def gradient(self, debiased: bool | None = None):
        """Envelope gradient of the last run w.r.t. X, Y, a, b (theta fixed)."""
        deb = self.debiased if debiased is None else bool(debiased)
        if deb and not self.debiased:
            raise ValueError("the debiased gradient needs a debiased run")
        if self.used_mode in ("recompute", "hybrid"):
            raise NotImplementedError("the adjoint reads the full stored features")
        if self.arccos is not None:
            raise NotImplementedError("the adjoint kernels differentiate the Gaussian map")
        dev = self.X.device
        gX = torch.empty_like(self.X)
        gY = torch.empty_like(self.Y)
        ga = torch.empty(self.x.n, dtype=torch.float32, device=dev)
        gb = torch.empty(self.y.n, dtype=torch.float32, device=dev)
        lsf_gradient(self.theta, self.x, self.y, self.s_xy, self.s_xx if deb else None,
                     self.s_yy if deb else None, self.results, deb, gX, gY, ga, gb,
                     self.stream, mode=self.used_mode)
        return gX, gY, ga, gb


    def anchor_gradient(self, debiased: bool | None = None, wrt: str = "U"):
        """Envelope gradient of the last run w.r.t. the anchors (q fixed).

        ``wrt="U"`` gives dW/dU (r x d); ``wrt="Z"`` gives dW/dZ = sigma dW/dU for
        the normal draws of U = sigma Z.
        """
        deb = self.debiased if debiased is None else bool(debiased)
        if deb and not self.debiased:
            raise ValueError("the debiased gradient needs a debiased run")
        if self.used_mode in ("recompute", "hybrid"):
            raise NotImplementedError("the adjoint reads the full stored features")
        if self.arccos is not None:
            raise NotImplementedError("the adjoint kernels differentiate the Gaussian map")
        if wrt not in ("U", "Z"):
            raise ValueError("wrt must be 'U' or 'Z'")
        th = self.theta
        gU = torch.empty((th.r, th.d), dtype=torch.float32, device=self.X.device)
        lsf_anchor_gradient(th, self.x, self.y, self.s_xy, self.s_xx if deb else None,
                            self.s_yy if deb else None, deb, gU, self.workspace,
                            scale=th.sigma if wrt == "Z" else 1.0, stream=self.stream,
                            mode=self.used_mode)
        return gU


def sinkhorn_divergence(X, Y, a, b, Z, eps: float, iters: int, debiased: bool = True,
                        mode: str = "stored") -> dict:
    """Solve once and return host scalars (W_xy, and W_xx, W_yy, W_bar if debiased)."""
    prob = SinkhornProblem(X, Y, a, b, Z, eps, mode=mode)
    prob.run(iters, debiased=debiased)
    return prob.values()


class SinkhornDivergenceFn(torch.autograd.Function):
    """W (or the debiased W_bar) as a differentiable function of X, Y, a, b and Z.

    theta (R, q, U) is computed from the inputs and then held fixed, as in the
    gradient formula after Prop. 3.3; the gradient w.r.t. Z (anchors U = sigma Z)
    moves the anchors with q fixed, as a learned feature map does. The backward
    pass uses the envelope gradient of the final iterate; no iteration is
    replayed.
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
        gZ = ctx.prob.anchor_gradient(wrt="Z") * g if ctx.needs_input_grad[4] else None
        return gX * g, gY * g, ga * g, gb * g, gZ, None, None, None


# ---------------------------------------------------------------- batched solver

def lsf_batch_plan(records, ldr: int, tile_bytes: int = 0, stream=None, mode: str = "stored"):
    """Plan a batch; returns (info, plan tensor). records: list of LsfBatchProblem."""
    arr = (LsfBatchProblem * len(records))(*records)
    info = LsfBatchInfo()
    check(lib().lsf_batch_plan(arr, len(records), int(ldr), MODES[mode], int(tile_bytes),
                               ctypes.byref(info), None, 0, _stream(stream)), "lsf_batch_plan")
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = torch.empty(info.plan_bytes + 256, dtype=torch.uint8, device=dev)
    off = (-buf.data_ptr()) % 256
    plan = buf[off:off + info.plan_bytes]
    check(lib().lsf_batch_plan(arr, len(records), int(ldr), MODES[mode], int(tile_bytes),
                               ctypes.byref(info), _p(plan), plan.numel(), _stream(stream)),
          "lsf_batch_plan")
    return info, plan


def lsf_solve_batched(info, plan, iters: int, stream=None) -> None:
    check(lib().lsf_solve_batched(ctypes.byref(info), _p(plan), int(iters), _stream(stream)),
          "lsf_solve_batched")


class _Batch:
    """One planned batch: problems (SinkhornProblem without scalings) in one mode."""

    def __init__(self, probs, ldr, mode, tile_bytes, stream):
        self.probs, self.ldr, self.mode, self.stream = probs, ldr, mode, stream
        dev = probs[0].X.device
        self.results = alloc_results(len(probs), dev)
        self.records = []
        for k, prob in enumerate(probs):
            s = Scalings.alloc(prob.x.n, prob.y.n, ldr, dev)
            prob.s_xy = s
            self.records.append(LsfBatchProblem(
                _p(prob.x.F).value, _p(prob.y.F).value, _p(prob.x.shift).value,
                _p(prob.y.shift).value, _p(prob.x.w).value, _p(prob.y.w).value, prob.x.n,
                prob.y.n, float(prob.eps), _p(s.u).value, _p(s.v).value, _p(s.t_u).value,
                _p(s.t_v).value, self.results.data_ptr() + k * RESULT_BYTES))
        if tile_bytes is None:
            from .autotune import best_batch_tile
            tile_bytes = best_batch_tile(self)
        self.tile_bytes = tile_bytes
        self.info, self.plan = lsf_batch_plan(self.records, ldr, tile_bytes, stream, mode=mode)
        self.graph = None

    @property
    def problems(self):
        return self.probs

    def run(self, iters):
        lsf_solve_batched(self.info, self.plan, iters, self.stream)

    def capture(self, iters):
        self.run(iters)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                lsf_solve_batched(self.info, self.plan, iters, s)
        self.graph = g


class BatchedSolver:
    """Many independent problems W(a_p, b_p), all sharing one feature width ldr.

    Builds each problem's theta and stored features (one launch per cloud), then
    solves all problems with the persistent batched kernel. ``problems``: list of
    objects with X, Y, a, b, Z (CUDA float32 tensors) and eps. ``tile_bytes=None``
    asks the autotuner.

    ``mode="auto"`` routes: ``route(iters)`` solves once in the scaling domain and
    moves the problems that reported a non-finite scaling into a second batch solved
    in the log domain; later runs solve both batches. ``mode="log"`` solves every
    problem in the log domain.
    """

    def __init__(self, problems, ldr: int | None = None, tile_bytes: int | None = None,
                 stream=None, mode: str = "stored"):
        self.stream = stream
        self.mode = mode
        rs = {int(p.Z.shape[0]) for p in problems}
        self.ldr = ldr if ldr is not None else ldr_for(max(rs))
        self.tile_bytes = tile_bytes
        first = "log" if mode == "log" else "stored"
        self.problems = [SinkhornProblem(p.X, p.Y, p.a, p.b, p.Z, p.eps, mode=first, ldr=self.ldr,
                                         stream=stream, scalings=False) for p in problems]
        for prob, p in zip(self.problems, problems):
            prob.eps = float(p.eps)
        self.batches = [(_Batch(self.problems, self.ldr, first, tile_bytes, stream),
                         list(range(len(self.problems))))]
        self.iters = None

    @property
    def info(self):
        return self.batches[0][0].info

    def route(self, iters: int) -> int:
        """Solve once; move range failures to a log-domain batch. Returns their number."""
        b0, idx0 = self.batches[0]
        b0.run(iters)
        bad = [k for k, v in zip(idx0, read_results(b0.results))
               if v["status"] & LSF_ERR_NONFINITE]
        if not bad:
            return 0
        good = [k for k in idx0 if k not in set(bad)]
        for k in bad:
            self.problems[k].switch_mode("log")
        batches = []
        if good:
            batches.append((_Batch([self.problems[k] for k in good], self.ldr, "stored",
                                   self.tile_bytes, self.stream), good))
        batches.append((_Batch([self.problems[k] for k in bad], self.ldr, "log", self.tile_bytes,
                               self.stream), bad))
        self.batches = batches
        return len(bad)

    def run(self, iters: int) -> None:
        self.iters = iters
        if self.mode == "auto" and len(self.batches) == 1 and self.batches[0][0].mode == "stored":
            self.route(iters)
        for b, _ in self.batches:
            b.run(iters)

    def capture(self, iters: int) -> None:
        """Capture each batch's solve (start, persistent kernel, reduction) in a CUDA graph."""
        self.run(iters)
        for b, _ in self.batches:
            b.capture(iters)
        self.iters = iters

    def replay(self) -> None:
        for b, _ in self.batches:
            b.graph.replay()

    def values(self) -> list[dict]:
        out = [None] * len(self.problems)
        for b, idx in self.batches:
            for k, v in zip(idx, read_results(b.results)):
                v["mode"] = b.mode
                out[k] = v
        return out


class MultiSinkhornProblem:
    """k pairs of weights (rows of A: k x n, B: k x m) on the same two clouds.

    One theta, one set of features (split into the bf16 pair planes of the
    tensor-core pass), and one multi-right-hand-side solve per term: every half
    iteration of Alg. 1 for all k pairs is two n x r x k contractions on the
    tensor cores. ``run(iters, debiased=True)`` also solves the self terms
    W(a_p, a_p) on (X, X) and W(b_p, b_p) on (Y, Y) with the same theta and
    combines Eq. (2) per pair. ``values`` returns, per pair, Eq. (6) (and
    Eq. (2)), the residual and the status, as a single solve of that pair
    reports them.
    """

    def __init__(self, X, Y, A, B, Z, eps: float, stream=None):
        for t in (X, Y, A, B, Z):
            _f32(t)
        if A.dim() != 2 or B.dim() != 2 or A.shape[0] != B.shape[0]:
            raise ValueError("A (k x n) and B (k x m) need the same number of rows")
        if A.shape[1] != X.shape[0] or B.shape[1] != Y.shape[0]:
            raise ValueError("A must have n columns and B m columns")
        self.stream = stream
        self.k = int(A.shape[0])
        dev = X.device
        n, d = X.shape
        m = Y.shape[0]
        r = Z.shape[0]
        R = float(lsf_radius(X, Y, stream=stream).item())
        q, sig = lsf_gaussian_params(R, eps, d)
        U, c = lsf_anchors(Z, q, sig, eps, stream=stream)
        self.theta = Theta(U, c, r, ldr_for(r), d, float(eps), R, q, sig)
        self.ldr2 = ldr2_for(r)
        Fx, self.shift_x = lsf_features(X, self.theta, stream=stream)
        Fy, self.shift_y = lsf_features(Y, self.theta, stream=stream)
        self.F2x = lsf_split_features(Fx, r, self.ldr2, stream=stream)
        self.F2y = lsf_split_features(Fy, r, self.ldr2, stream=stream)
        del Fx, Fy
        self.A, self.B = A, B
        self.n, self.m = n, m
        self.debiased = False
        kp = multi_kp(self.k)

        def scal(a, b):
            z = lambda *s_: torch.zeros(s_, dtype=torch.float32, device=dev)  # noqa: E731
            return {"U": z(self.k, a), "V": z(self.k, b), "Tu": z(kp, self.ldr2), "Tv": z(kp, self.ldr2)}

        self._scal = scal
        self.s = {"xy": scal(n, m)}
        self.U, self.V = self.s["xy"]["U"], self.s["xy"]["V"]
        self.Tu, self.Tv = self.s["xy"]["Tu"], self.s["xy"]["Tv"]
        self.results = alloc_results(self.k, dev)
        self.res = {"xy": self.results}
        nbytes = lsf_multi_workspace_bytes(self.ldr2, self.k)
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        off = (-ws.data_ptr()) % 256
        self.workspace = ws[off:off + nbytes]

    def _term(self, which: str):
        x = (self.F2x, self.shift_x, self.A) if which in ("xy", "xx") else (self.F2y, self.shift_y, self.B)
        y = (self.F2y, self.shift_y, self.B) if which in ("xy", "yy") else (self.F2x, self.shift_x, self.A)
        return x, y

    def run(self, iters: int, debiased: bool = False) -> None:
        """Launch the k solves (of each term of Eq. (2) when debiased) and their
        reductions on the stream (asynchronous); Eq. (2) is formed on the device."""
        self.debiased = bool(debiased)
        dev = self.A.device
        if not self.debiased:
            x, y = self._term("xy")
            s = self.s["xy"]
            lsf_solve_multi(self.theta, self.ldr2, x[0], x[1], x[2], y[0], y[1], y[2], iters,
                            s["U"], s["V"], s["Tu"], s["Tv"], self.res["xy"], self.workspace,
                            self.stream)
            return
        for t in ("xx", "yy"):
            if t not in self.s:
                x, y = self._term(t)
                self.s[t] = self._scal(x[2].shape[1], y[2].shape[1])
        if getattr(self, "res3", None) is None:
            self.res3 = alloc_results(3 * self.k, dev)
            self.wbar = torch.zeros(self.k, dtype=torch.float64, device=dev)
        lsf_multi_debiased(self.theta, self.ldr2, self.F2x, self.shift_x, self.A, self.F2y,
                           self.shift_y, self.B, iters, self.s["xy"], self.s["xx"], self.s["yy"],
                           self.res3, self.wbar, self.workspace, self.stream)

    def values(self) -> list[dict]:
        """Per pair: W (Eq. (6)), residual, status, iters, and with ``debiased``
        W_xx, W_yy and W_bar (Eq. (2), formed on the device) (synchronises)."""
        if not self.debiased:
            xy = read_results(self.res["xy"])
            return [{"W": r["W"], "residual": r["residual"], "status": r["status"],
                     "iters": r["iters"], "log_scale": r["log_scale"]} for r in xy]
        recs = read_results(self.res3)
        k = self.k
        wbar = self.wbar.cpu().tolist()
        out = []
        for p in range(k):
            a_, b_, c_ = recs[p], recs[k + p], recs[2 * k + p]
            out.append({"W": a_["W"], "residual": a_["residual"], "status": a_["status"],
                        "iters": a_["iters"], "log_scale": a_["log_scale"], "W_xx": b_["W"],
                        "W_yy": c_["W"], "res_xx": b_["residual"], "res_yy": c_["residual"],
                        "W_bar": wbar[p]})
        return out
