"""Write the oracle's values for the tiny two-mixture workload to tiny.json.

Calls only the FP64 oracle and the seeded input generator; nothing here comes
from the CUDA path.  Workload: 1000 + 1000 points in R^2 from a 3-component
mixture (std 0.3), the second cloud moved by +1; uniform weights; eps = 0.5;
r = 100 Gaussian features (Lemma 1); 100 iterations of Alg. 1; seed 0.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import oracle as o  # noqa: E402


def main():
    p = synth.tiny_problem(seed=0)
    out = o.divergence(p.X, p.Y, p.a, p.b, p.Z, p.eps, p.iters, debiased=True)
    th = out["theta"]
    rec = {
        "workload": p.name,
        "seed": 0,
        "R": th.R, "q": th.q, "sigma": th.sigma,
        "W_xy": out["W_xy"], "W_xx": out["W_xx"], "W_yy": out["W_yy"], "W_bar": out["W_bar"],
        "res_xy": out["res_xy"], "res_xx": out["res_xx"], "res_yy": out["res_yy"],
    }
    with open(os.path.join(HERE, "tiny.json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    main()
