"""Parity at the full workload sizes, in the launch configuration bench.py
uses, on outputs the oracle can compute one by one (sampled nodes), plus
properties that hold at any size (the adjoint identity, finite values).

Workloads: d=2 M=256 N=2^20 (m = 4, 6, 8; both methods), d=3 M=128 N=2^23
radial spokes (m = 6), d=2 M=512 N=4e6 batch 8 (m = 6) with gradients.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import oracle_plan, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nb = pytest.importorskip("paper_2502_07155_gb300")

N_SAMPLE = 3000


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_07155_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def sample_idx(N, n=N_SAMPLE, seed=0):
    return np.sort(np.random.default_rng(seed).choice(N, size=min(n, N), replace=False))


def adjoint_identity(plan, fh_d, g_d):
    f = plan.forward(fh_d)
    h = plan.adjoint(g_d)
    lhs = torch.vdot(g_d.reshape(-1).to(torch.complex128), f.reshape(-1).to(torch.complex128))
    rhs = torch.vdot(h.reshape(-1).to(torch.complex128), fh_d.reshape(-1).to(torch.complex128))
    return float(abs(lhs - rhs) / abs(lhs))


@pytest.mark.parametrize("m", [4, 6, 8])
@pytest.mark.parametrize("method", ["shannon", "classic"])
def test_d2_M256_N2e20(m, method):
    d, M, N = 2, 256, 1 << 20
    plan = nb.Plan(d, M, 2.0, m, precision="f32", method=method)
    x = W.nodes_uniform(N, d)
    fh = W.fhat_gaussian(M, d, dtype=np.complex64)
    g = W.adjoint_input(N, dtype=np.complex64)
    plan.set_nodes(to_dev(x))
    f = to_host(plan.forward(to_dev(fh)))
    idx = sample_idx(N)
    op = oracle_plan(plan)
    ref = O.forward(op, fh, x[idx])
    assert rel_l2(f[:, idx], ref) < 1e-5
    assert adjoint_identity(plan, to_dev(fh), to_dev(g)) < 1e-5
    if method == "shannon":
        # accuracy against the trigonometric sum on feasible sampled nodes
        feas = idx[W.feasible_mask(x[idx], m, 2 * M)][:1000]
        err = rel_l2(f[:, feas], O.ndft(fh, x[feas]))
        bound = {4: 6e-4, 6: 2e-5, 8: 1e-6}[m]
        assert err < bound, err


def test_d3_M128_N2e23_spokes():
    d, M, m = 3, 128, 6
    plan = nb.Plan(d, M, 2.0, m, precision="f32")
    x = W.nodes_spokes()
    N = x.shape[0]
    fh = W.fhat_gaussian(M, d, dtype=np.complex64)
    g = W.adjoint_input(N, dtype=np.complex64)
    plan.set_nodes(to_dev(x))
    f = to_host(plan.forward(to_dev(fh)))
    assert np.all(np.isfinite(f))
    # samples: uniform over the nodes plus the dense centre
    idx = np.unique(np.concatenate([sample_idx(N, 2000), np.argsort(np.abs(x).max(axis=1))[:500]]))
    op = oracle_plan(plan)
    ref = O.forward(op, fh, x[idx])
    assert rel_l2(f[:, idx], ref) < 1e-5
    assert adjoint_identity(plan, to_dev(fh), to_dev(g)) < 1e-5
    # adjoint at the densest cells: spread the samples' inputs only and compare
    plan.set_nodes(to_dev(x[idx]))
    gs = g[:, idx]
    h = to_host(plan.adjoint(to_dev(gs)))
    assert rel_l2(h, O.adjoint(op, gs, x[idx])) < 1e-5


def test_d2_M512_N4e6_B8_gradients():
    from paper_2502_07155_gb300.autograd import nfft_bandlimited
    d, M, m, N, B = 2, 512, 6, 4_000_000, 8
    plan = nb.Plan(d, M, 2.0, m, precision="f32", batch=B)
    x_np = W.nodes_uniform(N, d)
    fh_np = W.fhat_gaussian(M, d, batch=B, envelope=False, dtype=np.complex64)
    gf_np = W.adjoint_input(N, batch=B, dtype=np.complex64)
    x = to_dev(x_np).requires_grad_(True)
    fh = to_dev(fh_np).requires_grad_(True)
    f = nfft_bandlimited(fh, x, plan)
    f.backward(to_dev(gf_np))
    idx = sample_idx(N, 400)
    op = oracle_plan(plan)
    fac = O.precorrection_factors(op)
    grid = O.grid_samples(op, fh_np, fac)
    # forward on samples
    assert rel_l2(to_host(f.detach())[:, idx], O.step3_short_sums(op, grid, x_np[idx])) < 1e-5
    # node gradient on samples vs the oracle's analytic gradient
    gx = to_host(x.grad)[idx]
    der = np.zeros((B, idx.size, d), dtype=np.complex128)
    xs = x_np[idx].astype(np.float64)
    per = [O.nfft_oracle._tap_weights(op, xs, t) for t in range(d)]
    for t in range(d):
        ws = [p[2] if s == t else p[1] for s, p in enumerate(per)]
        wt = O.nfft_oracle._weight_tensor(ws)
        for b in range(B):
            vals = O.nfft_oracle._gather_tensor(grid[b], [p[0] for p in per])
            der[b, :, t] = np.sum(vals * wt, axis=(1, 2))
    ref_gx = np.sum(np.real(np.conj(gf_np[:, idx])[:, :, None] * der), axis=0)
    assert rel_l2(gx, ref_gx) < 1e-4
    # central differences (h = 1e-4 / L in FP64, one Richardson step) on the oracle's map
    v = W.fd_directions(idx.size, d)

    def phi(xx):
        return float(np.real(np.vdot(gf_np[:, idx], O.step3_short_sums(op, grid, xx))))
    h = 1e-4 / plan.L[0]
    cd = lambda hh: (phi(xs + hh * v) - phi(xs - hh * v)) / (2 * hh)
    rich = (4 * cd(h / 2) - cd(h)) / 3
    assert abs(np.sum(gx * v) - rich) <= 1e-4 * abs(rich)
    # gradient with respect to fhat: the adjoint, checked by the identity at full size
    lhs = torch.vdot(to_dev(gf_np).reshape(-1).to(torch.complex128), f.detach().reshape(-1).to(torch.complex128))
    rhs = torch.vdot(fh.grad.reshape(-1).to(torch.complex128), fh.detach().reshape(-1).to(torch.complex128))
    assert float(abs(lhs - rhs) / abs(lhs)) < 1e-5
