"""The oracle reproduces its stored values for the tiny two-mixture workload.

tests/golden/tiny.json is written by tests/golden/make_golden.py, which calls
only the oracle; this guards against an unnoticed change of its arithmetic.
"""
import json
import os

import synth
from oracle import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny.json")


def test_oracle_reproduces_tiny_golden():
    with open(GOLDEN) as f:
        g = json.load(f)
    p = synth.tiny_problem(seed=g["seed"])
    out = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=True)
    for k in ("W_xy", "W_xx", "W_yy", "W_bar"):
        assert abs(out[k] - g[k]) <= 1e-12 * max(1.0, abs(g[k])), k
    assert abs(out["theta"].q - g["q"]) < 1e-14
    for k in ("res_xy", "res_xx", "res_yy"):
        assert abs(out[k] - g[k]) < 1e-13
