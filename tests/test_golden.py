"""The stored oracle values for the tiny TV instance still reproduce (guards
against silent drift in the oracle or the input generators)."""
import json
import os

import numpy as np

from oracle import admm
from paper_2006_08303_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "tiny_tv_oracle.json")


def test_tiny_tv_golden():
    g = json.load(open(GOLD))
    P = inputs.tiny_tv()
    S = admm.analysis_setup(P.h, P.y, P.prior, P.lam, P.rho, P.beta)
    x, t, u, _ = admm.run_analysis(S, g["iters"])
    assert abs(np.linalg.norm(x) - g["x_norm"]) < 1e-10 * g["x_norm"]
    for m, a, b, v in g["x_samples"]:
        assert abs(x[m, a, b] - v) < 1e-10
