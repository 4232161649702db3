"""Failure detection on the GPU, without a GPU fault (through the C ABI).

Two kinds of failure are made on purpose, both from the host:

* bad data: an infinite coordinate makes the Lemma 1 radius infinite, which
  the host-side parameter check rejects (LSF_ERR_ARG) before any solve. A NaN
  in the points (which the radius, a maximum, passes over) or in the weights
  reaches the features or the scalings, and the solve reports LSF_ERR_NONFINITE
  in its device status, in every solver variant. Nothing hangs and the device
  stays usable.
* a bounded wait that runs out: the batched solver's test hook makes its
  consumers wait for a round flag that nothing sets, with a 20 ms limit. Every
  problem must then carry LSF_ERR_TIMEOUT, the launch must end within seconds
  (the kernel drains its copies in flight and returns), and the next batch,
  with the hook reset, must solve normally.
"""
import time

import numpy as np
import pytest
import torch

import synth
from oracle import oracle as o

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]


@pytest.fixture(scope="module")
def lsf():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2006_07057_gb300 as m
    m.lib()
    yield m
    m.lsf_set_batch_fault(4_000_000_000, 0)


def _dev(p):
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    return c(p.X), c(p.Y), c(p.a), c(p.b), c(p.Z)


def test_infinite_point_is_rejected_by_the_parameter_check(lsf):
    p = synth.small_problem(71, 500, 400, 3, 128, 0.3, 10)
    X, Y, a, b, Z = _dev(p)
    X[17, 1] = float("inf")
    with pytest.raises(lsf.LsfError) as e:
        lsf.SinkhornProblem(X, Y, a, b, Z, p.eps)
    assert e.value.status == lsf.LSF_ERR_ARG


@pytest.mark.parametrize("mode", ["stored", "hybrid", "auto"])
def test_nan_point_gives_a_nonfinite_status(lsf, mode):
    p = synth.small_problem(71, 500, 400, 3, 128, 0.3, 10)
    X, Y, a, b, Z = _dev(p)
    X[17, 1] = float("nan")
    prob = lsf.SinkhornProblem(X, Y, a, b, Z, p.eps, mode=mode)
    prob.run(p.iters, debiased=True)
    assert prob.values()["status"] & lsf.LSF_ERR_NONFINITE


@pytest.mark.parametrize("mode", ["stored", "recompute", "log", "hybrid"])
@pytest.mark.parametrize("where", ["points", "weights"])
def test_nan_reaches_the_device_status(lsf, mode, where):
    p = synth.small_problem(72, 3000, 2500, 3, 256, 0.3, 15)
    X, Y, a, b, Z = _dev(p)
    clean = lsf.SinkhornProblem(X, Y, a, b, Z, p.eps, mode=mode)
    if where == "points":
        X2 = X.clone()
        X2[123, 0] = float("nan")
        prob = lsf.SinkhornProblem(X2, Y, a, b, Z, p.eps, mode=mode, theta=clean.theta)
    else:
        a2 = a.clone()
        a2[77] = float("nan")
        prob = lsf.SinkhornProblem(X, Y, a2, b, Z, p.eps, mode=mode, theta=clean.theta)
    prob.run(p.iters, debiased=True)
    v = prob.values()
    # the three solves of Eq. (2) run in lock-step and report their status jointly
    assert all(r["status"] & lsf.LSF_ERR_NONFINITE for r in v["records"]), v["records"]
    # the device still works: the clean problem solves normally
    clean.run(p.iters, debiased=False)
    assert clean.values()["status"] == 0


class _P:
    def __init__(self, p):
        self.X, self.Y, self.a, self.b, self.Z = _dev(p)
        self.eps = p.eps


def test_batched_wait_runs_out_and_reports_timeout(lsf):
    probs = [synth.small_problem(80 + i, n, m, 3, 128, 0.4, 10, weights="dirichlet")
             for i, (n, m) in enumerate([(20000, 18000), (3000, 5000), (700, 900), (40000, 30000)])]
    solver = lsf.BatchedSolver([_P(p) for p in probs], tile_bytes=32 * 1024)
    assert solver.info.strategy == 0
    lsf.lsf_set_batch_fault(20_000_000, 1)
    try:
        t0 = time.monotonic()
        solver.run(10)
        torch.cuda.synchronize()
        took = time.monotonic() - t0
    finally:
        lsf.lsf_set_batch_fault(4_000_000_000, 0)
    vals = solver.values()
    assert all(v["status"] & lsf.LSF_ERR_TIMEOUT for v in vals), [v["status"] for v in vals]
    assert took < 30.0, took
    # the device and the solver are usable again: a normal run matches the oracle
    solver.run(10)
    for v, p in zip(solver.values(), probs):
        ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=False)
        assert v["status"] == 0, v
        assert abs(v["W"] - ref["W_xy"]) <= 1e-4 * abs(ref["W_xy"])
        assert abs(v["residual"] - ref["res_xy"]) <= 1e-5


def test_batch_fault_hook_validates_its_arguments(lsf):
    with pytest.raises(lsf.LsfError):
        lsf.lsf_set_batch_fault(5, 0)
    with pytest.raises(lsf.LsfError):
        lsf.lsf_set_batch_fault(4_000_000_000, 2)
