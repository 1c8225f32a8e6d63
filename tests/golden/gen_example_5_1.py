"""Write tests/golden/example_5_1.json from the oracle alone.

Example 5.1 (Section 5): d = 1, f(x) = sinc^2(M pi x / 2) with
fhat(v) = (2/M)(1 - |2v/M|), scaled Chebyshev nodes
x_j = cos((j-1) pi / N)(1/2 - m/L) with N = M/2, m = 5, lambda = 1
(L = 2M), sinh window; the error is max_j |f_j - f(x_j)| (Eq. 5.5).
The paper's figure (Fig. 5.2) is not printed, so these are the oracle's
values under the readings stated in the oracle, kept as regression data.

Run:  python tests/golden/gen_example_5_1.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

CITATION = "Example 5.1 and Fig. 5.2 (Section 5): M in {20,40,...,1000}, N = M/2, m = 5, lambda = 1, sinh window"


def errors(M, m=5):
    L = 2 * M
    x = W.nodes_chebyshev(M // 2, m, L)
    fh = (2.0 / M) * W.triangle(M, 1)[None].astype(complex)
    exact = O.sinc(M * np.pi * x[:, 0] / 2) ** 2
    out = {}
    for meth in ("shannon", "classic"):
        p = O.make_plan(1, M, 2.0, m, method=meth)
        out[meth] = float(np.max(np.abs(O.forward(p, fh, x)[0] - exact)))
    out["ndft"] = float(np.max(np.abs(O.ndft(fh, x)[0] - exact)))
    return out


if __name__ == "__main__":
    Ms = [20, 40, 80, 100, 200, 400, 600, 800, 1000]
    data = {"citation": CITATION, "m": 5, "lambda": 1, "window": "sinh",
            "beta_shannon": "pi*m*(1-1/sigma)", "beta_classic": "2*pi*m*(1-1/(2 sigma))",
            "M": Ms, "errors": {str(M): errors(M) for M in Ms}}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "example_5_1.json"), "w") as fh:
        json.dump(data, fh, indent=1)
