"""Continuous-batching server for debiased Sinkhorn divergence requests.

Requests of uneven shape (n, m, d, r, eps) arrive over time. The server keeps
each admitted request's features and scalings resident on the device, admits
waiting requests whenever a slot and enough of the HBM budget are free, and runs
every admitted request on its own CUDA stream, so the kernels of requests that
arrived while others were running overlap on the GPU (small requests occupy few
SMs). Completion is detected by polling CUDA events; the latency of a request is
its completion time minus its arrival time.

Each request runs exactly the single-problem path (lsf_features, lsf_debiased),
so its result does not depend on what else is running: the kernels reduce in
a fixed order for a given shape. A request whose scaling-domain run reports a
non-finite scaling (features or scalings outside the FP32 range) is run again
in the log domain in the same slot, found at completion time, so the scheduler
never blocks on it.

The plain competitor, `serve_sequential`, takes the same requests in arrival
order and solves them one at a time on one stream.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import LSF_ERR_NONFINITE, SinkhornProblem, ldr_for, lsf_workspace_bytes


@dataclass
class Request:
    """One divergence request: host arrays (FP32), eps, iterations and arrival time."""

    rid: int
    X: np.ndarray
    Y: np.ndarray
    a: np.ndarray
    b: np.ndarray
    Z: np.ndarray
    eps: float
    iters: int
    arrival_s: float = 0.0
    # filled by the server
    start_s: float = 0.0
    done_s: float = 0.0
    W_bar: float = float("nan")
    status: int = -1
    result: dict = field(default_factory=dict)

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def request_bytes(n: int, m: int, r: int, d: int) -> int:
    """Device bytes a request holds while admitted (features, points, scalings, workspace)."""
    ldr = ldr_for(r)
    feats = 4 * (n + m) * ldr
    pts = 4 * (n + m) * (d + 2) + 4 * r * (d + 1) + 4 * r * d
    scal = 4 * (2 * n + 2 * m + (n + m)) + 4 * 6 * ldr
    return feats + pts + scal + lsf_workspace_bytes(ldr) + 4096


class _Slot:
    def __init__(self, device):
        self.stream = torch.cuda.Stream(device=device)
        self.req = None
        self.prob = None
        self.mode = "stored"
        self.host_out = torch.empty(1, dtype=torch.float64).pin_memory()
        self.done = torch.cuda.Event()
        self.bytes = 0


class Server:
    """Admit-by-budget continuous batching over CUDA streams."""

    def __init__(self, budget_bytes: float = 40e9, slots: int = 16, device=None):
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.budget = float(budget_bytes)
        self.in_use = 0.0
        self.slots = [_Slot(self.device) for _ in range(slots)]
        self.peak_bytes = 0.0
        self.peak_inflight = 0
        self.relaunched = 0

    def _launch(self, slot: _Slot, req: Request, now: float, mode: str = "stored") -> None:
        slot.req = req
        slot.mode = mode
        if mode == "stored":
            req.start_s = now
        with torch.cuda.stream(slot.stream):
            t = {k: torch.from_numpy(getattr(req, k)).pin_memory().to(self.device, non_blocking=True)
                 for k in ("X", "Y", "a", "b", "Z")}
            prob = SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], req.eps, mode=mode,
                                   stream=slot.stream)
            prob.run(req.iters, debiased=True)
            slot.host_out.copy_(prob.wbar, non_blocking=True)
            slot.done.record(slot.stream)
        slot.prob = prob

    def _finish(self, slot: _Slot, now: float):
        """Finish the slot's request, or relaunch it in the log domain (returns None)."""
        req = slot.req
        vals = slot.prob.values()
        if (vals["status"] & LSF_ERR_NONFINITE) and slot.mode == "stored":
            self.relaunched += 1
            self._launch(slot, req, now, mode="log")
            return None
        req.done_s = now
        req.W_bar = float(slot.host_out.item())
        req.status = vals["status"]
        req.result["mode"] = slot.mode
        req.result.update({k: vals[k] for k in ("W_xy", "W_xx", "W_yy", "res_xy") if k in vals})
        self.in_use -= slot.bytes
        slot.req = None
        slot.prob = None
        slot.bytes = 0
        return req

    def serve(self, requests: list[Request], realtime: bool = True) -> list[Request]:
        """Serve requests in arrival order; returns them with timings and results.

        With ``realtime`` the arrival times are honoured against the wall clock
        (a request cannot start before it arrives); otherwise all are present at
        time 0.
        """
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting: collections.deque = collections.deque()
        finished = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        if not realtime:
            for r in pending:
                r.arrival_s = 0.0
        while pending or waiting or any(s.req is not None for s in self.slots):
            tnow = now()
            while pending and pending[0].arrival_s <= tnow:
                waiting.append(pending.popleft())
            # completions
            for s in self.slots:
                if s.req is not None and s.done.query():
                    r = self._finish(s, now())
                    if r is not None:
                        finished.append(r)
            # admissions: first come, first served, as budget and slots allow
            while waiting:
                req = waiting[0]
                need = request_bytes(req.X.shape[0], req.Y.shape[0], req.Z.shape[0], req.X.shape[1])
                free = next((s for s in self.slots if s.req is None), None)
                if free is None:
                    break
                if self.in_use + need > self.budget and self.in_use > 0:
                    break
                waiting.popleft()
                free.bytes = need
                self.in_use += need
                self.peak_bytes = max(self.peak_bytes, self.in_use)
                self._launch(free, req, now())
                self.peak_inflight = max(self.peak_inflight, sum(s.req is not None for s in self.slots))
            if not waiting and pending and all(s.req is None for s in self.slots):
                # idle until the next arrival
                dt = pending[0].arrival_s - now()
                if dt > 0:
                    time.sleep(min(dt, 0.01))
            else:
                time.sleep(0)
        return finished


def serve_sequential(requests: list[Request], realtime: bool = True, device=None) -> list[Request]:
    """The plain competitor: one request at a time, in arrival order, one stream."""
    device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    reqs = sorted(requests, key=lambda r: r.arrival_s)
    host_out = torch.empty(1, dtype=torch.float64).pin_memory()
    t0 = time.perf_counter()
    if not realtime:
        for r in reqs:
            r.arrival_s = 0.0
    for req in reqs:
        wait = req.arrival_s - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        req.start_s = time.perf_counter() - t0
        t = {k: torch.from_numpy(getattr(req, k)).pin_memory().to(device, non_blocking=True)
             for k in ("X", "Y", "a", "b", "Z")}
        prob = SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], req.eps, mode="auto")
        prob.run(req.iters, debiased=True)
        host_out.copy_(prob.wbar, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        req.done_s = time.perf_counter() - t0
        req.W_bar = float(host_out.item())
        req.status = prob.values()["status"]
    return reqs


def latency_stats(reqs: list[Request]) -> dict:
    lat = np.sort(np.array([r.latency_s for r in reqs]))
    span = max(r.done_s for r in reqs) - min(r.arrival_s for r in reqs)
    pick = lambda q: float(lat[min(len(lat) - 1, int(q * len(lat)))])  # noqa: E731
    return {"requests": len(reqs), "throughput_per_s": len(reqs) / span if span > 0 else None,
            "latency_ms_p50": 1e3 * pick(0.5), "latency_ms_p99": 1e3 * pick(0.99),
            "latency_ms_max": 1e3 * float(lat[-1]), "span_s": span}
