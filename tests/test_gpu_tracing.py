"""NVTX tracing levels leave the results alone (GPU).

The ranges are host-side markers around entry points (level 1) and kernel
launches (level 2); a solve at every level must give the same bits.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_tracing_levels_do_not_change_results():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2006_07057_gb300 as lsf
    lsf.lib()
    p = synth.small_problem(61, 3000, 2000, 3, 256, 0.3, 20, weights="dirichlet")
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
    out = {}
    prev = lsf.lsf_set_tracing(1)
    try:
        for level in (0, 1, 2):
            lsf.lsf_set_tracing(level)
            for mode in ("stored", "hybrid"):
                prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode=mode)
                prob.run(p.iters, debiased=True)
                g = prob.values()
                assert g["status"] == 0
                out[(level, mode)] = (g["W_bar"], g["res_xy"])
    finally:
        lsf.lsf_set_tracing(prev)
    for mode in ("stored", "hybrid"):
        assert out[(0, mode)] == out[(1, mode)] == out[(2, mode)]
