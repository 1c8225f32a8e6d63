"""Parity at the full workload sizes, in the launch configuration bench.py
uses, on outputs the oracle can compute one by one (sampled nodes, selected
grid cells), element by element over the whole grid where the oracle
finishes in seconds, plus properties that hold at any size (the adjoint
identity, finite values).

Workloads: d=2 M=256 N=2^20 (m = 4, 6, 8; both methods; FP32 and FP64),
d=3 M=128 N=2^23 radial spokes (m = 6 and 8; FP32 and FP64), d=2 M=512
N=4e6 batch 8 (m = 6) with gradients.
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
    assert rel_l2(gx, ref_gx) < 1e-5
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


# --------------------------------------------------------------------------- element-wise adjoint at full size

TOL = {"f64": 1e-12, "f32": 1e-5, "f32c": 1e-5}


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_d2_M256_N2e20_adjoint_elementwise(prec):
    """The whole transposed short-sum grid Psi^T g (512^2 cells) and the
    whole adjoint D F^H Psi^T g (256^2 coefficients) of all 2^20 nodes at
    m = 8, element by element against the oracle."""
    d, M, m, N = 2, 256, 8, 1 << 20
    rdt, cdt = (np.float64, np.complex128) if prec == "f64" else (np.float32, np.complex64)
    plan = nb.Plan(d, M, 2.0, m, precision=prec)
    x = W.nodes_uniform(N, d, dtype=rdt)
    g = W.adjoint_input(N, dtype=cdt)
    plan.set_nodes(to_dev(x))
    h = to_host(plan.adjoint(to_dev(g)))
    plan.spread_grid(to_dev(g))
    u = plan.grid()
    op = oracle_plan(plan)
    u_ref = O.adjoint_short_sums(op, g, x)
    assert rel_l2(u, u_ref) < TOL[prec]
    fac = O.precorrection_factors(op)
    h_ref = O.adjoint_idft(op, u_ref) * fac[0][None, :, None] * fac[1][None, None, :]
    assert rel_l2(h, h_ref) < TOL[prec]


def test_d2_M256_N2e20_f64_forward_sampled():
    """FP64 forward of all 2^20 nodes at m = 8, sampled nodes against the
    oracle at the FP64 tolerance."""
    d, M, m, N = 2, 256, 8, 1 << 20
    plan = nb.Plan(d, M, 2.0, m, precision="f64")
    x = W.nodes_uniform(N, d, dtype=np.float64)
    fh = W.fhat_gaussian(M, d, dtype=np.complex128)
    plan.set_nodes(to_dev(x))
    f = to_host(plan.forward(to_dev(fh)))
    idx = sample_idx(N)
    assert rel_l2(f[:, idx], O.forward(oracle_plan(plan), fh, x[idx])) < TOL["f64"]


def spoke_cell_blocks(L, m, T=8):
    """Grid cells (storage indices) for the spoke workload: the 2x2x2 cells
    at the centre where every spoke meets (the densest cells), 2x2x2 cells
    straddling tile boundaries in the sparse part (several boxes of the
    ordered flush cover them), the grid's first and last cells (zero
    extension at the edge of I_L) and a few single cells."""
    h = L // 2
    blocks = [
        [(h - 1 + a, h - 1 + b, h - 1 + c) for a in (0, 1) for b in (0, 1) for c in (0, 1)],
        [(3 * T - 1 + a, 5 * T - 1 + b, 2 * T - 1 + c) for a in (0, 1) for b in (0, 1) for c in (0, 1)],
        [(L - 4 * T - 1 + a, h + T - 1 + b, L - 2 * T - 1 + c) for a in (0, 1) for b in (0, 1) for c in (0, 1)],
        [(0, 0, 0), (L - 1, L - 1, L - 1), (1, h, L - 2)],
        [(h + 40, h - 30, h + 5), (h - 7, h + 9, h + 2)],
    ]
    return [np.array(b, dtype=np.int64) for b in blocks]


def nodes_reaching(x, cells, L, m):
    """Indices of the nodes whose taps can reach any of the cells."""
    lo = cells.min(axis=0) - L // 2 - m - 1
    hi = cells.max(axis=0) - L // 2 + m + 1
    u = L * x.astype(np.float64)
    return np.flatnonzero(np.all((u >= lo) & (u <= hi), axis=1))


@pytest.mark.parametrize("m,prec", [(6, "f32c"), (8, "f32c"), (6, "f64")])
def test_d3_M128_N2e23_spread_cells(m, prec):
    """Transposed short sums of all 2^23 spoke nodes (no re-binning: the
    full-density runs, long same-cell runs at the centre, many items per
    tile) at selected cells against the oracle's definition evaluated from
    the nodes that reach them; then the sampled forward."""
    d, M = 3, 128
    rdt, cdt = (np.float64, np.complex128) if prec == "f64" else (np.float32, np.complex64)
    plan = nb.Plan(d, M, 2.0, m, precision=prec)
    x = W.nodes_spokes().astype(rdt)
    N = x.shape[0]
    g = W.adjoint_input(N, dtype=cdt)
    plan.set_nodes(to_dev(x))
    _, _, off = plan.binning()
    assert np.diff(off.astype(np.int64)).max() > 4 * 1024     # the centre tiles hold several work items
    plan.spread_grid(to_dev(g))
    grid = plan.grid_tensor()
    op = oracle_plan(plan)
    L = plan.L[0]
    got_all, ref_all = [], []
    for cells in spoke_cell_blocks(L, m):
        sel = nodes_reaching(x, cells, L, m)
        ref = O.adjoint_short_sums_at(op, g[:, sel], x[sel], cells)
        idx = torch.from_numpy(cells).cuda()
        got = to_host(grid[0, idx[:, 0], idx[:, 1], idx[:, 2]])[None, :]
        if np.linalg.norm(ref) > 0:
            assert rel_l2(got, ref) < TOL[prec], (cells[0], sel.size)
        else:
            assert np.all(got == 0)
        got_all.append(got)
        ref_all.append(ref)
    assert rel_l2(np.concatenate(got_all, axis=1), np.concatenate(ref_all, axis=1)) < TOL[prec]
    fh = W.fhat_gaussian(M, d, dtype=cdt)
    f = to_host(plan.forward(to_dev(fh)))
    idx = np.unique(np.concatenate([sample_idx(N, 1500), np.argsort(np.abs(x).max(axis=1))[:300]]))
    assert rel_l2(f[:, idx], O.forward(op, fh, x[idx])) < TOL[prec]
