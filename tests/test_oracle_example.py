"""Example 5.1 (Section 5) on the oracle.

The paper's Fig. 5.2 is a placeholder, so its values are not available:
this checks what the mathematics fixes -- with exact samples fhat(k) at
integer k both algorithms approximate the trigonometric sum (the NDFT, a
rectangle-rule quadrature of Eq. 1.1), so each one's deviation from the
NDFT stays at its own window-error level -- and that the oracle still
reproduces the regression values its committed generator wrote.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "example_5_1.json")))


@pytest.mark.parametrize("M", [20, 100, 400, 1000])
def test_example_5_1(M):
    m = 5
    L = 2 * M
    x = W.nodes_chebyshev(M // 2, m, L)
    fh = (2.0 / M) * W.triangle(M, 1)[None].astype(complex)
    exact = O.sinc(M * np.pi * x[:, 0] / 2) ** 2
    nd = O.ndft(fh, x)[0]
    errs = {}
    for meth in ("shannon", "classic"):
        p = O.make_plan(1, M, 2.0, m, method=meth)
        f = O.forward(p, fh, x)[0]
        errs[meth] = np.max(np.abs(f - exact))
        # deviation from the trigonometric sum: window error only
        # (sum |fhat| = 1 here; e^{-beta} of each window bounds the scale)
        beta = O.default_beta(meth, m, 2.0)
        assert np.max(np.abs(f - nd)) < 20 * np.exp(-beta)
    ref = GOLD["errors"][str(M)]
    for meth in ("shannon", "classic"):
        assert errs[meth] == pytest.approx(ref[meth], rel=1e-9)
    # the quadrature (periodisation) error of the NDFT is the common floor
    assert np.max(np.abs(nd - exact)) == pytest.approx(ref["ndft"], rel=1e-9)
