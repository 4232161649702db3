"""The C-ABI library builds, loads without a GPU and exports every declared symbol.

Host-only entry points (Lemma 1 parameters) and host-side argument checks are
exercised here; nothing in this file launches a kernel.
"""
import ctypes
import math

import pytest

import paper_2006_07057_gb300 as lsf
from paper_2006_07057_gb300 import _binding as B
from oracle import oracle as o


def test_library_exports_every_header_symbol():
    L = lsf.lib()
    names = B.header_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(names) <= set(B._SIGNATURES), set(names) - set(B._SIGNATURES)


def test_version_and_empty_error():
    assert lsf.lsf_version() == 2
    assert isinstance(lsf.lib().lsf_last_error(), bytes)


@pytest.mark.parametrize("R,eps,d", [(0.0, 0.5, 2), (1e-6, 0.5, 2), (2.76, 0.5, 2),
                                     (1.73, 0.1, 3), (14.5, 1.0, 128), (3.0, 0.05, 16),
                                     (50.0, 0.01, 3)])
def test_gaussian_params_match_oracle(R, eps, d):
    q, s = lsf.lsf_gaussian_params(R, eps, d)
    qo, so = o.gaussian_params(R, eps, d)
    assert abs(q - qo) <= 1e-14 * qo and abs(s - so) <= 1e-14 * so


@pytest.mark.parametrize("args", [(1.0, 0.0, 2), (1.0, -1.0, 2), (1.0, 0.5, 0), (-1.0, 0.5, 2),
                                  (math.inf, 0.5, 2), (math.nan, 0.5, 2)])
def test_gaussian_params_rejects_bad_arguments(args):
    with pytest.raises(B.LsfError) as e:
        lsf.lsf_gaussian_params(*args)
    assert e.value.status == B.LSF_ERR_ARG


def test_device_entry_points_validate_before_launching():
    L = lsf.lib()
    th = B.LsfTheta(None, None, 0, 4, 2, 0.5)
    cl = B.LsfCloud(None, None, None, None, 0)
    sc = B.LsfScalings(None, None, None, None)
    rc = L.lsf_solve(ctypes.byref(th), ctypes.byref(cl), ctypes.byref(cl), 10, 0,
                     ctypes.byref(sc), None, None, 0, None)
    assert rc == B.LSF_ERR_ARG
    assert b"r >= 1" in L.lsf_last_error()
    th = B.LsfTheta(None, None, 8, 6, 2, 0.5)   # ldr not a multiple of 4
    rc = L.lsf_solve(ctypes.byref(th), ctypes.byref(cl), ctypes.byref(cl), 10, 0,
                     ctypes.byref(sc), None, None, 0, None)
    assert rc in (B.LSF_ERR_ARG, B.LSF_ERR_UNSUPPORTED)
    th = B.LsfTheta(None, None, 8, 8, 2, 0.5)
    rc = L.lsf_solve(ctypes.byref(th), ctypes.byref(cl), ctypes.byref(cl), 10, 0,
                     ctypes.byref(sc), None, None, 0, None)
    assert rc == B.LSF_ERR_ARG and b"n >= 1" in L.lsf_last_error()
    assert L.lsf_radius(None, 1, None, 1, 2, None, None) == B.LSF_ERR_ARG
    assert L.lsf_features(None, 1, None, None, None, None, None) == B.LSF_ERR_ARG
    assert L.lsf_workspace_bytes(6, None) == B.LSF_ERR_ARG
    b = ctypes.c_size_t()
    assert L.lsf_workspace_bytes(2048, ctypes.byref(b)) == B.LSF_ERR_UNSUPPORTED


def test_ldr_rounding():
    assert [lsf.ldr_for(r) for r in (1, 3, 4, 100, 1023, 1024)] == [4, 4, 4, 100, 1024, 1024]


def test_hybrid_column_split_is_host_only():
    # half of the float4 column groups (rounded down) are stored; the rest rebuilt
    assert [lsf.lsf_hybrid_columns(ldr) for ldr in (8, 12, 100, 256, 1020, 1024)] == \
        [4, 8, 52, 128, 512, 512]
    for bad in (4, 6, 1028):
        with pytest.raises(B.LsfError) as e:
            lsf.lsf_hybrid_columns(bad)
        assert e.value.status == B.LSF_ERR_UNSUPPORTED


def test_tracing_level_switch():
    # host-only: the level is a process-wide switch read at each entry point
    assert lsf.lsf_set_tracing(2) == 1          # the default is entry-point ranges
    assert lsf.lsf_set_tracing(0) == 2
    for bad in (-1, 3):
        with pytest.raises(B.LsfError) as e:
            lsf.lsf_set_tracing(bad)
        assert e.value.status == B.LSF_ERR_ARG
    assert lsf.lsf_set_tracing(1) == 0


def test_tolerance_solves_validate_before_launching():
    # the stopping-rule arguments are checked on the host, before any device work
    L = lsf.lib()
    th = B.LsfTheta(None, None, 8, 8, 2, 0.5)
    cl = B.LsfCloud(None, None, None, None, 0)
    sc = B.LsfScalings(None, None, None, None)
    for max_iters, tol, k in ((0, 1e-3, 5), (10, -1.0, 5), (10, float("nan"), 5), (10, 1e-3, 0)):
        rc = L.lsf_solve_tol(ctypes.byref(th), ctypes.byref(cl), ctypes.byref(cl), max_iters, tol, k,
                             0, ctypes.byref(sc), None, None, 0, None)
        assert rc == B.LSF_ERR_ARG, (max_iters, tol, k)
        rc = L.lsf_debiased_tol(ctypes.byref(th), ctypes.byref(cl), ctypes.byref(cl), max_iters, tol, k,
                                0, ctypes.byref(sc), ctypes.byref(sc), ctypes.byref(sc), None, None,
                                None, 0, None)
        assert rc == B.LSF_ERR_ARG, (max_iters, tol, k)
    # valid stopping arguments: the empty cloud is the next thing refused
    rc = L.lsf_solve_tol(ctypes.byref(th), ctypes.byref(cl), ctypes.byref(cl), 10, 1e-3, 5, 0,
                         ctypes.byref(sc), None, None, 0, None)
    assert rc == B.LSF_ERR_ARG and b"n >= 1" in L.lsf_last_error()
