"""Continuous-batching server: results alone vs in the mix, overlap, budget (GPU).

Each admitted request runs the single-problem path on its own stream; the
kernels reduce in a fixed order for a given shape, so a request's divergence is
the same whether it runs alone or overlapped with others. The tolerance stated
for the divergence (1e-4 relative to |W_xy| + |W_xx|/2 + |W_yy|/2) is checked,
and in practice the values agree bit for bit.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2006_07057_gb300 as m
    m.lib()
    from paper_2006_07057_gb300 import serve as s
    return s


def requests(serve, count, seed=0, n_hi=1 << 12, iters=30):
    out = []
    for i, rq in enumerate(synth.serving_stream(seed=seed, count=count, rate_per_s=4000.0,
                                                iters=iters, n_lo=1 << 8, n_hi=n_hi)):
        p = rq.problem
        out.append(serve.Request(i, p.X, p.Y, p.a, p.b, p.Z, p.eps, iters, rq.arrival_s))
    return out


def test_results_same_alone_and_in_the_mix(serve):
    reqs = requests(serve, 24)
    alone = serve.serve_sequential([serve.Request(r.rid, r.X, r.Y, r.a, r.b, r.Z, r.eps, r.iters)
                                    for r in reqs], realtime=False)
    srv = serve.Server(budget_bytes=20e9, slots=8)
    mixed = srv.serve(reqs, realtime=False)
    assert srv.peak_inflight > 1, "requests did not overlap"
    by_id = {r.rid: r for r in alone}
    for r in mixed:
        a = by_id[r.rid]
        assert r.status == 0 and a.status == 0
        scale = abs(r.result["W_xy"]) + 0.5 * abs(r.result["W_xx"]) + 0.5 * abs(r.result["W_yy"])
        assert abs(r.W_bar - a.W_bar) <= 1e-4 * scale, (r.rid, r.W_bar, a.W_bar)


def test_admission_respects_the_budget(serve):
    reqs = requests(serve, 16, seed=1)
    biggest = max(serve.request_bytes(r.X.shape[0], r.Y.shape[0], r.Z.shape[0], r.X.shape[1])
                  for r in reqs)
    budget = 2.5 * biggest
    srv = serve.Server(budget_bytes=budget, slots=8)
    done = srv.serve(reqs, realtime=False)
    assert len(done) == len(reqs)
    assert srv.peak_bytes <= budget
    stats = serve.latency_stats(done)
    assert stats["latency_ms_p99"] >= stats["latency_ms_p50"] > 0


def test_batching_server_matches_alone_and_the_oracle(serve):
    # the continuous-batching server solves each request's three terms as rows of
    # a batched problem table; the result must match the request solved alone
    # (sequential arm) and the oracle at the divergence tolerance
    from oracle import oracle as o
    reqs = requests(serve, 20, seed=3)
    alone = serve.serve_sequential([serve.Request(r.rid, r.X, r.Y, r.a, r.b, r.Z, r.eps, r.iters)
                                    for r in reqs], realtime=False)
    srv = serve.BatchingServer(budget_bytes=20e9, max_group=8)
    mixed = srv.serve(reqs, realtime=False)
    assert len(mixed) == len(reqs)
    assert srv.groups_run >= 3 and srv.peak_inflight > 1
    by_id = {r.rid: r for r in alone}
    for r in mixed:
        a = by_id[r.rid]
        assert r.status == 0 and a.status == 0, (r.rid, r.status, a.status)
        scale = abs(r.result["W_xy"]) + 0.5 * abs(r.result["W_xx"]) + 0.5 * abs(r.result["W_yy"])
        assert abs(r.W_bar - a.W_bar) <= 1e-4 * scale, (r.rid, r.W_bar, a.W_bar)
    for r in mixed[:4]:
        ref = o.divergence(r.X, r.Y, r.a, r.b, r.Z, r.eps, r.iters, debiased=True)
        scale = abs(ref["W_xy"]) + 0.5 * abs(ref["W_xx"]) + 0.5 * abs(ref["W_yy"])
        assert abs(r.W_bar - ref["W_bar"]) <= 1e-4 * scale


def test_batching_server_routes_range_failures_to_the_log_domain(serve):
    # small eps with d = 16 puts some requests outside the FP32 range of the
    # scaling domain; they are re-admitted in a log-domain group
    out = []
    for i, rq in enumerate(synth.serving_stream(seed=5, count=12, rate_per_s=4000.0, iters=30,
                                                n_lo=1 << 8, n_hi=1 << 11)):
        p = rq.problem
        out.append(serve.Request(i, p.X, p.Y, p.a, p.b, p.Z, 0.05, 30, rq.arrival_s))
    alone = serve.serve_sequential([serve.Request(r.rid, r.X, r.Y, r.a, r.b, r.Z, r.eps, r.iters)
                                    for r in out], realtime=False)
    srv = serve.BatchingServer(budget_bytes=10e9, max_group=6)
    mixed = srv.serve(out, realtime=False)
    by_id = {r.rid: r for r in alone}
    for r in mixed:
        a = by_id[r.rid]
        assert r.status == 0 and a.status == 0, (r.rid, r.status, a.status)
        scale = abs(r.result["W_xy"]) + 0.5 * abs(r.result["W_xx"]) + 0.5 * abs(r.result["W_yy"])
        assert abs(r.W_bar - a.W_bar) <= 1e-4 * scale, (r.rid, r.W_bar, a.W_bar)
    if any(a.result["mode"] == "log" for a in alone):
        assert srv.relaunched > 0 and any(r.result["mode"] == "log" for r in mixed)


def test_server_runs_large_low_dimensional_requests_on_the_hybrid_pass(serve):
    # requests past the one-launch solver's size with d <= 4 start on the hybrid
    # pass (serve.first_mode); the sequential arm routes the same way, and both
    # must match the oracle
    from oracle import oracle as o
    out = []
    for i, rq in enumerate(synth.serving_stream(seed=11, count=40, rate_per_s=4000.0, iters=20,
                                                n_lo=1 << 15, n_hi=1 << 15)):
        p = rq.problem
        if p.X.shape[1] <= 3 and p.Z.shape[0] == 512 and p.eps >= 0.2:
            out.append(serve.Request(len(out), p.X, p.Y, p.a, p.b, p.Z, p.eps, 20, rq.arrival_s))
        if len(out) == 2:
            break
    assert len(out) == 2
    assert all(serve.first_mode(r) == "hybrid" for r in out)
    alone = serve.serve_sequential([serve.Request(r.rid, r.X, r.Y, r.a, r.b, r.Z, r.eps, r.iters)
                                    for r in out], realtime=False)
    srv = serve.Server(budget_bytes=20e9, slots=4)
    mixed = srv.serve(out, realtime=False)
    by_id = {r.rid: r for r in alone}
    for r in mixed:
        a = by_id[r.rid]
        assert r.status == 0 and a.status == 0
        assert r.result["mode"] == "hybrid" and a.result["mode"] == "hybrid"
        # (the scaling-domain oracle: eps >= 0.2 at d = 2 is well inside FP64 range)
        ref = o.divergence(r.X, r.Y, r.a, r.b, r.Z, r.eps, r.iters, debiased=True, mode="scaled")
        scale = abs(ref["W_xy"]) + 0.5 * abs(ref["W_xx"]) + 0.5 * abs(ref["W_yy"])
        assert abs(r.W_bar - ref["W_bar"]) <= 1e-4 * scale, (r.rid, r.W_bar, ref["W_bar"])
        assert abs(r.W_bar - a.W_bar) <= 1e-4 * scale
