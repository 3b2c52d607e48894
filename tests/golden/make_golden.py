"""Writes tests/golden/tiny_tv_oracle.json from the FP64 oracle only.

The paper prints no worked numerical example, so the stored values here are
the oracle's own, for the 64x64x3 anisotropic-TV instance (lambda=1e-2, rho=1,
beta=1, 50 iterations of Alg. 1).  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import admm  # noqa: E402
from paper_2006_08303_gb300 import inputs  # noqa: E402


def main():
    P = inputs.tiny_tv()
    S = admm.analysis_setup(P.h, P.y, P.prior, P.lam, P.rho, P.beta)
    x, t, u, hist = admm.run_analysis(S, P.iters, keep_history=True)
    rng = np.random.default_rng(0)
    idx = [(int(m), int(a), int(b)) for m, a, b in zip(rng.integers(0, P.M, 16), rng.integers(0, P.N, 16),
                                                        rng.integers(0, P.N, 16))]
    out = {
        "source": "oracle.admm.run_analysis on inputs.tiny_tv() (seed 20060830)",
        "iters": P.iters,
        "x_norm": float(np.linalg.norm(x)),
        "u_norm": float(np.linalg.norm(u)),
        "x_samples": [[m, a, b, float(x[m, a, b])] for m, a, b in idx],
        "r_rel": [h.r_rel for h in hist],
        "s_rel": [h.s_rel for h in hist],
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_tv_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
