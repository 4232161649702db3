"""The whole-path entry point and the library's automatic domain choice (GPU).

lsf_pipeline_run takes host arrays and returns host values; everything between
(radius, Lemma 1 parameters with the Lambert W0 evaluated on the device,
anchors, features, Alg. 1 for each term, Eq. (6) and Eq. (2)) runs on the
device in one caller arena. It is checked against the FP64 oracle at the
parity tolerances (divergence 1e-4 relative, residual 1e-5 absolute), its
Lemma 1 parameters against the oracle's to 1e-6 relative (R is the FP32 norm
of an FP32 point), and against the resident-problem path it must agree with.

LSF_MODE_AUTO is driven through the C ABI on problems inside and outside the
FP32 range of the scaling domain: the result record must say which domain
produced W, and W must match the oracle either way.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import oracle as o

pytestmark = pytest.mark.gpu

W_RTOL = 1e-4
RES_ATOL = 1e-5


@pytest.fixture(scope="module")
def lsf():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2006_07057_gb300 as m
    m.lib()
    return m


def host(p):
    return [torch.from_numpy(np.ascontiguousarray(getattr(p, k))).pin_memory() for k in "XYabZ"]


def check_against_oracle(out, ref, debiased, res_rtol=0.0):
    assert out["status"] == 0, out
    assert abs(out["W_xy"] - ref["W_xy"]) <= W_RTOL * abs(ref["W_xy"]), (out["W_xy"], ref["W_xy"])
    assert abs(out["residual_xy"] - ref["res_xy"]) <= RES_ATOL + res_rtol * ref["res_xy"]
    if debiased:
        scale = abs(ref["W_xy"]) + 0.5 * abs(ref["W_xx"]) + 0.5 * abs(ref["W_yy"])
        assert abs(out["W"] - ref["W_bar"]) <= W_RTOL * scale, (out["W"], ref["W_bar"])
        for k in ("xx", "yy"):
            assert abs(out[f"residual_{k}"] - ref[f"res_{k}"]) <= RES_ATOL + res_rtol * ref[f"res_{k}"]
    else:
        assert out["W"] == out["W_xy"]


@pytest.mark.parametrize("mode", ["stored", "recompute", "hybrid", "log", "auto"])
@pytest.mark.parametrize("debiased", [False, True])
def test_pipeline_matches_oracle(lsf, mode, debiased):
    p = synth.small_problem(61, 3001, 2003, 3, 300, 0.3, 30, weights="dirichlet")
    hp = lsf.HostPipeline()
    hp.run(*host(p), p.eps, p.iters, debiased=debiased, mode=mode)
    out = hp.result()
    ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=debiased)
    th = ref["theta"]
    assert abs(out["R"] - th.R) <= 1e-6 * th.R
    assert abs(out["q"] - th.q) <= 1e-6 * th.q
    assert abs(out["sigma"] - th.sigma) <= 1e-6 * th.sigma
    assert out["iters"] == p.iters
    assert out["mode_name"] == ("stored" if mode == "auto" else mode)
    check_against_oracle(out, ref, debiased)


def test_pipeline_agrees_with_the_resident_path_and_reuses_its_arena(lsf):
    hp = lsf.HostPipeline()
    for seed, n, m, r in ((62, 5000, 4000, 256), (63, 700, 900, 128)):   # second one smaller
        p = synth.small_problem(seed, n, m, 2, r, 0.5, 25, weights="dirichlet")
        hp.run(*host(p), p.eps, p.iters, debiased=True, mode="stored")
        out = hp.result()
        t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
        prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps)
        prob.run(p.iters, debiased=True)
        g = prob.values()
        scale = abs(g["W_xy"]) + 0.5 * abs(g["W_xx"]) + 0.5 * abs(g["W_yy"])
        # the device and host Lambert W0 may differ in the last bits of q
        assert abs(out["W"] - g["W_bar"]) <= 1e-6 * scale
        assert abs(out["residual_xy"] - g["res_xy"]) <= 1e-7


def test_pipeline_large_workload_shape(lsf):
    p = synth.large_problem(seed=0, n=1 << 13)
    hp = lsf.HostPipeline()
    hp.run(*host(p), p.eps, p.iters, debiased=True, mode="hybrid")
    out = hp.result()
    check_against_oracle(out, o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=True,
                                           mode="scaled"), True)


HARD = [(16, 0.05, 1.0, 17), (3, 0.05, 1.0, 19)]


@pytest.mark.parametrize("d,eps,shift,seed", HARD)
def test_auto_routes_range_failures_to_the_log_domain(lsf, d, eps, shift, seed):
    p = synth.small_problem(seed, 400, 300, d, 128, eps, 40, weights="dirichlet", shift=shift)
    ref = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=True)
    th = ref["theta"]
    spread = max(float(np.ptp(o.log_features(P, th.U, p.eps, th.q), axis=1).max()) for P in (p.X, p.Y))
    hp = lsf.HostPipeline()
    hp.run(*host(p), p.eps, p.iters, debiased=True, mode="stored")
    stored = hp.result()
    hp.run(*host(p), p.eps, p.iters, debiased=True, mode="auto")
    out = hp.result()
    if stored["status"] & lsf.LSF_ERR_NONFINITE:
        assert out["mode_name"] == "log"
    else:
        assert out["mode_name"] == "stored"
    check_against_oracle(out, ref, True, res_rtol=2.0 * spread * 2.0 ** -23)


def test_auto_through_the_debiased_entry_point(lsf):
    # the C call itself: lsf_debiased(LSF_MODE_AUTO) fills F and shift, picks the
    # domain, and records it in every result record
    p = synth.small_problem(17, 400, 300, 16, 128, 0.05, 40, weights="dirichlet", shift=1.0)
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda() for k in "XYabZ"}
    prob = lsf.SinkhornProblem(t["X"], t["Y"], t["a"], t["b"], t["Z"], p.eps, mode="auto")
    prob.run(p.iters, debiased=True)
    recs = lsf.read_results(prob.results)
    assert len({r["mode"] for r in recs}) == 1
    assert prob.used_mode in ("stored", "log")
    assert lsf.lib().lsf_version() == 2


def test_pipeline_rejects_bad_descriptions_and_small_arenas(lsf):
    L = lsf.lib()
    b = ctypes.c_size_t()
    # (iters = 0 only prepares, which the stored and log modes allow)
    for bad in (lsf.pipeline_desc(0, 10, 2, 8, 0.5, 3), lsf.pipeline_desc(10, 10, 2, 8, -1.0, 3),
                lsf.pipeline_desc(10, 10, 2, 8, 0.5, -1), lsf.pipeline_desc(10, 10, 2, 8, 0.5, 0,
                                                                           mode="hybrid")):
        assert L.lsf_pipeline_bytes(ctypes.byref(bad), ctypes.byref(b)) == lsf.LSF_ERR_ARG
    desc = lsf.pipeline_desc(10, 10, 2, 2000, 0.5, 3)
    assert L.lsf_pipeline_bytes(ctypes.byref(desc), ctypes.byref(b)) == lsf.LSF_ERR_UNSUPPORTED
    p = synth.small_problem(5, 50, 40, 2, 16, 0.5, 3)
    desc = lsf.pipeline_desc(50, 40, 2, 16, 0.5, 3)
    need = lsf.lsf_pipeline_bytes(desc)
    arena = lsf.alloc_arena(need - 256, torch.device("cuda", 0))
    out = torch.zeros(ctypes.sizeof(lsf.LsfPipelineOut), dtype=torch.uint8).pin_memory()
    with pytest.raises(lsf.LsfError) as e:
        lsf.lsf_pipeline_run(desc, *host(p), arena, out.data_ptr())
    assert e.value.status == lsf.LSF_ERR_WORKSPACE
