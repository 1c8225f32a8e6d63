"""The paper's numerical experiments (Section 5) run through the library.

* Example 5.1 (Fig. 5.2): f(x) = sinc^2(M pi x / 2), whose Fourier transform
  is the triangle (2/M)(1 - |2v/M|) on [-M/2, M/2]; scaled Chebyshev nodes
  x_j = cos((j-1) pi / N)(1/2 - m/L), N = M/2, m = 5, L = 2M; the error is
  max_j |f_j - f(x_j)| (Eq. 5.5), for Algorithm 4.2 and for the classical
  NFFT (Algorithm 2.1) on the same samples fhat(k), k in I_M.
* Fig. 5.1: e(v) = max_p |exp(2 pi i v x_p) - h(x_p)| (Eq. 5.3) for
  v_s = -M/2 - m + s/S, s = 0..S(M + 2m), at P equispaced points of an
  interval, with h the short sums of exp(2 pi i v l / L) against psi (the
  approximation of Section 5 with D = I, |I_L| psi_hat ~ 1) or against the
  periodic phi divided by L phi_hat(v) (the classical NFFT).  All values of
  v are one batched interpolation (batch = number of v).

Nothing here evaluates the transform itself: the grids go through
interp_grid / forward of a plan.
"""
from __future__ import annotations

import time

import numpy as np

import workloads as W

from . import Plan


def example51_errors(M: int, m: int = 5, precision: str = "f64", method: str = "shannon",
                     beta: float | None = None, precorrect: bool = True) -> float:
    """max_j |f_j - sinc^2(M pi x_j / 2)| of one forward transform (d = 1,
    sigma = 2) on the N = M/2 scaled Chebyshev nodes of Example 5.1."""
    import torch
    L = 2 * M
    x = W.nodes_chebyshev(M // 2, m, L)
    fh = ((2.0 / M) * W.triangle(M, 1)).astype(np.complex128)[None]
    rdt = torch.float64 if precision == "f64" else torch.float32
    cdt = torch.complex128 if precision == "f64" else torch.complex64
    plan = Plan(1, M, 2.0, m, precision=precision, method=method, beta=beta, precorrect=precorrect)
    plan.set_nodes(torch.from_numpy(x).to("cuda", rdt))
    f = plan.forward(torch.from_numpy(fh).to("cuda", cdt)).to(torch.complex128).cpu().numpy()[0]
    plan.close()
    exact = np.sinc(M * x[:, 0] / 2) ** 2          # np.sinc(t) = sin(pi t)/(pi t)
    return float(np.max(np.abs(f - exact)))


def fig51_frequencies(M: int = 20, m: int = 5, S: int = 32) -> np.ndarray:
    """v_s = -M/2 - m + s/S, s = 0..S(M + 2m)."""
    return -M / 2 - m + np.arange(S * (M + 2 * m) + 1, dtype=np.float64) / S


def fig51_errors(M: int = 20, m: int = 5, S: int = 32, P: int = 100_000, interval: str = "full",
                 method: str = "shannon", beta: float | None = None, precision: str = "f64"):
    """e(v) of Fig. 5.1 on the GPU.  interval: 'full' ([-1/2, 1/2)) or
    'trunc' ([-1/2 + m/L, 1/2 - m/L)).  Returns (v, e, seconds of the
    batched interpolation)."""
    import torch
    L = 2 * M
    v = fig51_frequencies(M, m, S)
    B = v.size
    lo, hi = (-0.5, 0.5) if interval == "full" else (-0.5 + m / L, 0.5 - m / L)
    x = lo + (hi - lo) * np.arange(P, dtype=np.float64) / P
    rdt = torch.float64 if precision == "f64" else torch.float32
    cdt = torch.complex128 if precision == "f64" else torch.complex64
    plan = Plan(1, M, 2.0, m, precision=precision, method=method, beta=beta, batch=B)
    xd = torch.from_numpy(x[:, None]).to("cuda", rdt)
    plan.set_nodes(xd)
    vd = torch.from_numpy(v).cuda()
    ell = torch.arange(-L // 2, L // 2, dtype=torch.float64, device="cuda")
    grid = torch.exp(2j * np.pi * vd[:, None] * ell[None, :] / L)          # centred index l + L/2
    if method == "classic":
        grid = grid / (L * plan.window_transform(vd))[:, None]
    plan.grid_tensor().copy_(grid.to(cdt))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = plan.interp_grid()
    plan.sync()
    seconds = time.perf_counter() - t0
    xs = xd[:, 0].to(torch.float64)
    e = torch.empty(B, dtype=torch.float64, device="cuda")
    for b0 in range(0, B, 64):                                              # bounded temporaries
        b1 = min(B, b0 + 64)
        ex = torch.exp(2j * np.pi * vd[b0:b1, None] * xs[None, :])
        e[b0:b1] = torch.max(torch.abs(ex - h[b0:b1].to(torch.complex128)), dim=1).values
    plan.close()
    return v, e.cpu().numpy(), seconds
