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
