"""The allocation-free solve agrees with the workspace solve (GPU).

lsf_solve_noalloc serves callers that cannot allocate device memory (a
framework pool that owns the device, a serving loop that must not block on the
allocator): it takes its scratch from a fixed array inside the library. Here it
is called through the C ABI twice in a row, and each result is compared with
lsf_solve run with a caller-provided workspace on the same inputs, at the
tolerances of the other parity tests (divergence 1e-4 relative, residual 1e-5
absolute).

The cases cover the multi-launch streamed passes, which use every region of the
scratch (per-CTA partial r-vectors, group partials, residual partials, arrival
counters): the stored pass with the single-launch small-problem solver switched
off, the recompute pass, the log-domain pass and the hybrid pass (at r = 256 and
at r = 1024, where its fixed-stride variant runs), plus the small-problem solver
itself. Running two solves in a row checks that the array's leftover contents
from one call do not leak into the next.

This file is collected last on purpose: if the built-in array were laid out
wrongly, a run that stops at the first failure has then already run every other
test.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,small,r", [("stored", 0, 256), ("recompute", 1, 256), ("log", 1, 256),
                                          ("stored", 1, 256), ("hybrid", 1, 256), ("hybrid", 1, 1024)])
def test_noalloc_solve_matches_workspace_solve_twice(mode, small, r):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2006_07057_gb300 as lsf
    p = synth.small_problem(21, 3001, 2503, 3, r, 0.3, 30, weights="dirichlet")
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode=mode)
    dev = t["X"].device

    def w_of(s, res):
        lsf.lsf_divergence(prob.theta, [prob.x], [prob.y], [s], [res], [1.0], None,
                           prob.workspace, mode=mode)
        return lsf.read_results(res)[0]

    lsf.lsf_set_small_solver(small)
    try:
        ref_s = lsf.Scalings.alloc(p.n, p.m, prob.theta.ldr, dev)
        ref_r = lsf.alloc_results(1, dev)
        lsf.lsf_solve(prob.theta, prob.x, prob.y, p.iters, mode, ref_s, ref_r, prob.workspace)
        ref = w_of(ref_s, ref_r)
        assert ref["status"] == 0
        for _ in range(2):
            s = lsf.Scalings.alloc(p.n, p.m, prob.theta.ldr, dev)
            r = lsf.alloc_results(1, dev)
            lsf.lsf_solve_noalloc(prob.theta, prob.x, prob.y, p.iters, mode, s, r)
            got = w_of(s, r)
            assert got["status"] == 0
            assert abs(got["W"] - ref["W"]) <= 1e-4 * abs(ref["W"])
            assert abs(got["residual"] - ref["residual"]) <= 1e-5
            if mode == "log":
                # log u~, log v~: absolute agreement
                assert torch.allclose(s.u, ref_s.u, rtol=0, atol=1e-4 * (1 + ref_s.u.abs().max().item()))
                assert torch.allclose(s.v, ref_s.v, rtol=0, atol=1e-4 * (1 + ref_s.v.abs().max().item()))
            else:
                assert torch.allclose(s.u, ref_s.u, rtol=1e-5, atol=0)
                assert torch.allclose(s.v, ref_s.v, rtol=1e-5, atol=0)
    finally:
        lsf.lsf_set_small_solver(1)
