"""Continuous-batching server for debiased Sinkhorn divergence requests.

Requests of uneven shape (n, m, d, r, eps) arrive over time. The server owns one
device pool the size of its HBM budget, carved first-fit into per-request
arenas, and a set of slots, each a CUDA stream with a pinned result record. A
waiting request is admitted as soon as a slot is free and its arena fits in the
pool; it then runs the whole path on its slot's stream with one library call
(lsf_pipeline_run: inputs copied in, Lemma 1 parameters and anchors on the
device, features, the lock-step solves of Eq. (2), the result record copied
out), so the kernels of requests that arrived while others were running overlap
on the GPU. Admission never waits on the device and allocates nothing;
completion is detected by polling CUDA events. The latency of a request is its
completion time minus its arrival time.

Each request runs exactly the single-problem path, so its result does not depend
on what else is running: the kernels reduce in a fixed order for a given shape.
A request whose scaling-domain run reports a non-finite scaling (features or
scalings outside the FP32 range) is run again in the log domain in the same
slot and arena, found at completion time, so the scheduler never blocks on it.

The plain competitor, `serve_sequential`, takes the same requests in arrival
order and solves them one at a time on one stream with the same call and the
same routing.
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (LSF_ERR_NONFINITE, MODE_NAMES, RESULT_BYTES, LsfBatchProblem, LsfPipelineOut, alloc_arena,
               ldr_for, lsf_batch_plan, lsf_pipeline_bytes, lsf_pipeline_finish, lsf_pipeline_layout,
               lsf_pipeline_run, lsf_solve_batched, pipeline_desc)


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
    host: list | None = None   # the inputs in pinned host memory (see pin)

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s

    def pin(self) -> "Request":
        """Hold the inputs in pinned host memory, as a server receiving requests into
        pinned buffers would; the copies to the device are then asynchronous."""
        if self.host is None:
            self.host = [torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).pin_memory()
                         for v in (self.X, self.Y, self.a, self.b, self.Z)]
        return self

    def desc(self, mode: str):
        return pipeline_desc(self.X.shape[0], self.Y.shape[0], self.X.shape[1], self.Z.shape[0],
                             self.eps, self.iters, True, mode)


HYBRID_MAX_D = 4
SMALL_SOLVER_ENTRIES = 1 << 24   # the library's default size rule for its one-launch solver


def first_mode(req: "Request") -> str:
    """The domain and pass a request starts in. The hybrid pass (half the feature
    columns rebuilt in registers, half streamed) beats the stored pass when its
    rebuilt entries are cheap (d + 3 FP32 operations each); for larger d the
    stored pass is faster. Requests whose three terms all fit the stored mode's
    one-launch solver ((n + m) ldr <= 2^24 entries for each) stay stored: their
    time is launches, not entries. A non-finite scaling in either sends the
    request to the log domain."""
    n, m, d = req.X.shape[0], req.Y.shape[0], req.X.shape[1]
    small = 2 * max(n, m) * ldr_for(req.Z.shape[0]) <= SMALL_SOLVER_ENTRIES
    return "hybrid" if d <= HYBRID_MAX_D and not small else "stored"


def request_bytes(n: int, m: int, r: int, d: int, mode: str = "stored") -> int:
    """Device bytes a request holds while admitted: its lsf_pipeline_run arena
    (inputs, theta, features, scalings, results, workspace)."""
    return lsf_pipeline_bytes(pipeline_desc(n, m, d, r, 1.0, 1, True, mode))


class FreeList:
    """First-fit allocation of 256-byte aligned ranges of [0, size) (host only)."""

    ALIGN = 256

    def __init__(self, nbytes: int):
        self.size = int(nbytes) // self.ALIGN * self.ALIGN
        self.free_list = [(0, self.size)] if self.size else []   # (offset, length), sorted, coalesced
        self.in_use = 0

    def alloc(self, nbytes: int):
        """(offset, length) of the first free range that fits, or None."""
        need = max(self.ALIGN, (int(nbytes) + self.ALIGN - 1) // self.ALIGN * self.ALIGN)
        for k, (off, ln) in enumerate(self.free_list):
            if ln >= need:
                if ln == need:
                    self.free_list.pop(k)
                else:
                    self.free_list[k] = (off + need, ln - need)
                self.in_use += need
                return off, need
        return None

    def free(self, off: int, ln: int) -> None:
        self.in_use -= ln
        fl = self.free_list
        k = 0
        while k < len(fl) and fl[k][0] < off:
            k += 1
        fl.insert(k, (off, ln))
        # coalesce with the neighbours
        if k + 1 < len(fl) and fl[k][0] + fl[k][1] == fl[k + 1][0]:
            fl[k] = (fl[k][0], fl[k][1] + fl[k + 1][1])
            fl.pop(k + 1)
        if k > 0 and fl[k - 1][0] + fl[k - 1][1] == fl[k][0]:
            fl[k - 1] = (fl[k - 1][0], fl[k - 1][1] + fl[k][1])
            fl.pop(k)


class Pool(FreeList):
    """A FreeList over one device buffer (the server's admission budget)."""

    def __init__(self, nbytes: int, device):
        super().__init__(nbytes)
        self.buf = alloc_arena(self.size, device)

    def view(self, off: int, ln: int) -> torch.Tensor:
        return self.buf[off:off + ln]


class _Slot:
    def __init__(self, device):
        self.stream = torch.cuda.Stream(device=device)
        self.out = torch.zeros(ctypes.sizeof(LsfPipelineOut), dtype=torch.uint8).pin_memory()
        self.done = torch.cuda.Event()
        self.req = None
        self.mode = "stored"
        self.range = None   # (offset, bytes) in the pool

    def record(self) -> dict:
        o = LsfPipelineOut.from_address(self.out.data_ptr())
        return {k: getattr(o, k) for k, _ in LsfPipelineOut._fields_ if k != "reserved"}


def _launch(req: Request, mode: str, arena: torch.Tensor, out: torch.Tensor, stream) -> None:
    req.pin()
    lsf_pipeline_run(req.desc(mode), *req.host, arena, out.data_ptr(), stream)


def _finished(req: Request, rec: dict, now: float) -> Request:
    req.done_s = now
    req.W_bar = rec["W"]
    req.status = rec["status"]
    req.result = {"mode": MODE_NAMES.get(rec["mode"], "?"), "W_xy": rec["W_xy"], "W_xx": rec["W_xx"],
                  "W_yy": rec["W_yy"], "res_xy": rec["residual_xy"], "R": rec["R"], "q": rec["q"]}
    return req


class Server:
    """Admit-by-budget continuous batching over CUDA streams, one device pool."""

    def __init__(self, budget_bytes: float = 40e9, slots: int = 16, device=None):
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.budget = float(budget_bytes)
        self.pool = Pool(int(budget_bytes), self.device)
        self.slots = [_Slot(self.device) for _ in range(slots)]
        self.peak_bytes = 0.0
        self.peak_inflight = 0
        self.relaunched = 0

    @property
    def in_use(self) -> float:
        return float(self.pool.in_use)

    def _start(self, slot: _Slot, req: Request, mode: str) -> None:
        slot.req = req
        slot.mode = mode
        _launch(req, mode, self.pool.view(*slot.range), slot.out, slot.stream)
        slot.done.record(slot.stream)

    def _finish(self, slot: _Slot, now: float):
        """Finish the slot's request, or relaunch it in the log domain (returns None)."""
        req = slot.req
        rec = slot.record()
        if (rec["status"] & LSF_ERR_NONFINITE) and slot.mode != "log":
            self.relaunched += 1
            self._start(slot, req, "log")
            return None
        _finished(req, rec, now)
        self.pool.free(*slot.range)
        slot.req = None
        slot.range = None
        return req

    def serve(self, requests: list[Request], realtime: bool = True) -> list[Request]:
        """Serve requests in arrival order; returns them with timings and results.

        With ``realtime`` the arrival times are honoured against the wall clock
        (a request cannot start before it arrives); otherwise all are present at
        time 0.
        """
        for r in requests:
            r.pin()
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
            # admissions: first come, first served, as slots and the pool allow
            while waiting:
                free = next((s for s in self.slots if s.req is None), None)
                if free is None:
                    break
                req = waiting[0]
                rng = self.pool.alloc(request_bytes(req.X.shape[0], req.Y.shape[0], req.Z.shape[0],
                                                    req.X.shape[1]))
                if rng is None:
                    if all(s.req is None for s in self.slots):
                        raise MemoryError(f"request {req.rid} does not fit the {self.budget:.3g}-byte budget")
                    break
                waiting.popleft()
                free.range = rng
                req.start_s = now()
                self._start(free, req, first_mode(req))
                self.peak_bytes = max(self.peak_bytes, float(self.pool.in_use))
                self.peak_inflight = max(self.peak_inflight, sum(s.req is not None for s in self.slots))
            if not waiting and pending and all(s.req is None for s in self.slots):
                # idle until the next arrival
                dt = pending[0].arrival_s - now()
                if dt > 0:
                    time.sleep(min(dt, 0.01))
            else:
                time.sleep(0)
        return finished


class _Group:
    """Requests admitted together: prepared, solved by one persistent batched launch
    per feature width, finished; one event marks the end of its work."""

    def __init__(self, reqs, mode, plans):
        self.reqs = reqs
        self.mode = mode
        self.plans = plans          # keeps the device plans alive while the group runs
        self.done = torch.cuda.Event()


class BatchingServer:
    """Continuous batching through the persistent batched solver.

    Waiting requests are admitted in groups whenever fewer than ``inflight``
    groups are on the GPU. Each admitted request gets an arena from the pool
    (first fit, the budget bounds the pool) and a pinned result record, and is
    prepared on the device (lsf_pipeline_run with iters = 0: inputs in, Lemma 1
    on the device, anchors, features). The three terms of Eq. (2) of every
    request of the group become rows of a device problem table (one
    lsf_batch_plan per feature width), which one cooperative persistent launch
    solves for all iterations (lsf_solve_batched); lsf_pipeline_finish then forms
    Eq. (2) per request and copies its record out. Requests that report a
    non-finite scaling go back to the head of the queue and are re-admitted in a
    log-domain group (log features, the batched solver's log mode). Admission
    does not wait on the device; the only host waits are the plan copies (small,
    on their own stream).
    """

    def __init__(self, budget_bytes: float = 40e9, max_group: int = 256, inflight: int = 2,
                 device=None):
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.budget = float(budget_bytes)
        self.pool = Pool(int(budget_bytes), self.device)
        self.max_group = int(max_group)
        self.inflight = int(inflight)
        self.stream = torch.cuda.Stream(device=self.device)
        self.plan_stream = torch.cuda.Stream(device=self.device)
        self.outs = torch.zeros((max_group * (inflight + 1), ctypes.sizeof(LsfPipelineOut)),
                                dtype=torch.uint8).pin_memory()
        self.free_outs = list(range(self.outs.shape[0]))
        self.peak_bytes = 0.0
        self.peak_inflight = 0
        self.relaunched = 0
        self.groups_run = 0

    def _admit(self, reqs: list, mode: str) -> _Group:
        st = self.stream
        by_ldr: dict = {}
        for r in reqs:
            desc = pipeline_desc(r.X.shape[0], r.Y.shape[0], r.X.shape[1], r.Z.shape[0], r.eps, 0,
                                 True, mode)
            r._desc = desc
            arena = self.pool.view(*r._range)
            v = lsf_pipeline_layout(desc, arena)
            recs = []
            for t, (cx, cy) in enumerate(((v.x, v.y), (v.x, v.x), (v.y, v.y))):
                sc = v.s[t]
                recs.append(LsfBatchProblem(cx.F, cy.F, cx.shift, cy.shift, cx.w, cy.w, cx.n, cy.n,
                                            float(r.eps), sc.u, sc.v, sc.t_u, sc.t_v,
                                            v.result + t * RESULT_BYTES))
            by_ldr.setdefault(ldr_for(r.Z.shape[0]), []).extend(recs)
        # the device problem tables, planned on their own stream (small host waits)
        plans = []
        for ldr, recs in sorted(by_ldr.items()):
            info, plan = lsf_batch_plan(recs, ldr, 0, self.plan_stream, mode=mode)
            plans.append((info, plan))
        # the group's work, in order, on the group stream
        for r in reqs:
            r.pin()
            lsf_pipeline_run(r._desc, *r.host, self.pool.view(*r._range), 0, st)
        iters = reqs[0].iters
        for info, plan in plans:
            lsf_solve_batched(info, plan, iters, st)
        for r in reqs:
            lsf_pipeline_finish(r._desc, self.pool.view(*r._range), self.outs[r._out].data_ptr(), st)
        g = _Group(reqs, mode, plans)
        g.done.record(st)
        self.groups_run += 1
        return g

    def serve(self, requests: list[Request], realtime: bool = True) -> list[Request]:
        """Serve requests in arrival order; returns them with timings and results."""
        if len({r.iters for r in requests}) > 1:
            raise ValueError("one iteration count per served stream (the batched solve shares it)")
        for r in requests:
            r.pin()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting: collections.deque = collections.deque()
        retry: collections.deque = collections.deque()   # range failures, arenas kept
        running: list = []
        finished = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        if not realtime:
            for r in pending:
                r.arrival_s = 0.0
        while pending or waiting or retry or running:
            tnow = now()
            while pending and pending[0].arrival_s <= tnow:
                waiting.append(pending.popleft())
            for g in [g for g in running if g.done.query()]:
                running.remove(g)
                t = now()
                for r in g.reqs:
                    o = LsfPipelineOut.from_address(self.outs[r._out].data_ptr())
                    rec = {k: getattr(o, k) for k, _ in LsfPipelineOut._fields_}
                    if (rec["status"] & LSF_ERR_NONFINITE) and g.mode == "stored":
                        self.relaunched += 1
                        retry.append(r)
                        continue
                    _finished(r, rec, t)
                    self.pool.free(*r._range)
                    self.free_outs.append(r._out)
                    finished.append(r)
            while len(running) < self.inflight and (retry or waiting):
                if retry:
                    group = [retry.popleft() for _ in range(min(len(retry), self.max_group))]
                    running.append(self._admit(group, "log"))
                    continue
                group = []
                while waiting and len(group) < self.max_group and self.free_outs:
                    r = waiting[0]
                    rng = self.pool.alloc(request_bytes(r.X.shape[0], r.Y.shape[0], r.Z.shape[0],
                                                        r.X.shape[1]))
                    if rng is None:
                        if not group and not running:
                            raise MemoryError(f"request {r.rid} does not fit the {self.budget:.3g}-byte budget")
                        break
                    waiting.popleft()
                    r._range = rng
                    r._out = self.free_outs.pop()
                    r.start_s = now()
                    group.append(r)
                if not group:
                    break
                running.append(self._admit(group, "stored"))
                self.peak_bytes = max(self.peak_bytes, float(self.pool.in_use))
                self.peak_inflight = max(self.peak_inflight, sum(len(g.reqs) for g in running))
            if not waiting and not retry and pending and not running:
                dt = pending[0].arrival_s - now()
                if dt > 0:
                    time.sleep(min(dt, 0.01))
            else:
                time.sleep(0)
        return finished


def serve_sequential(requests: list[Request], realtime: bool = True, device=None) -> list[Request]:
    """The plain competitor: one request at a time, in arrival order, one stream, the
    same library call and the same routing as ``Server`` (``first_mode``, then the
    log domain after a non-finite run)."""
    device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    reqs = sorted(requests, key=lambda r: r.arrival_s)
    for r in reqs:
        r.pin()
    arena = alloc_arena(max(request_bytes(r.X.shape[0], r.Y.shape[0], r.Z.shape[0], r.X.shape[1])
                            for r in reqs), device)
    out = torch.zeros(ctypes.sizeof(LsfPipelineOut), dtype=torch.uint8).pin_memory()
    stream = torch.cuda.current_stream(device)
    t0 = time.perf_counter()
    if not realtime:
        for r in reqs:
            r.arrival_s = 0.0
    for req in reqs:
        wait = req.arrival_s - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        req.start_s = time.perf_counter() - t0
        for mode in (first_mode(req), "log"):
            _launch(req, mode, arena, out, stream)
            stream.synchronize()
            rec = LsfPipelineOut.from_address(out.data_ptr())
            rec = {k: getattr(rec, k) for k, _ in LsfPipelineOut._fields_}
            if not (rec["status"] & LSF_ERR_NONFINITE):
                break
        _finished(req, rec, time.perf_counter() - t0)
    return reqs


def latency_stats(reqs: list[Request]) -> dict:
    lat = np.sort(np.array([r.latency_s for r in reqs]))
    span = max(r.done_s for r in reqs) - min(r.arrival_s for r in reqs)
    pick = lambda q: float(lat[min(len(lat) - 1, int(q * len(lat)))])  # noqa: E731
    return {"requests": len(reqs), "throughput_per_s": len(reqs) / span if span > 0 else None,
            "latency_ms_p50": 1e3 * pick(0.5), "latency_ms_p99": 1e3 * pick(0.99),
            "latency_ms_max": 1e3 * float(lat[-1]), "span_s": span}
