"""Gradients of the differentiable transform (autograd.Function over the
C-ABI): torch.autograd.gradcheck in FP64, central differences with a
Richardson step, and the oracle's analytic gradient."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import oracle_plan, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nb = pytest.importorskip("paper_2502_07155_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_07155_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("d,M,method", [(1, 16, "shannon"), (2, 8, "shannon"), (2, 8, "classic")])
def test_gradcheck_fp64(d, M, method):
    from paper_2502_07155_gb300.autograd import NFFTBL
    plan = nb.Plan(d, M, 2.0, 3, precision="f64", method=method, batch=2)
    x = to_dev(W.nodes_uniform(12, d, dtype=np.float64, seed=3)).requires_grad_(True)
    fh = to_dev(W.fhat_gaussian(plan.M, batch=2, dtype=np.complex128)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b: NFFTBL.apply(a, b, plan), (fh, x), eps=1e-7, atol=1e-6, rtol=1e-5)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_autograd_matches_oracle_gradient(prec, tol):
    from paper_2502_07155_gb300.autograd import nfft_bandlimited
    d, M, m, N, B = 2, 32, 5, 600, 3
    cdt = np.complex128 if prec == "f64" else np.complex64
    rdt = np.float64 if prec == "f64" else np.float32
    plan = nb.Plan(d, M, 2.0, m, precision=prec, batch=B)
    x_np = W.nodes_uniform(N, d, dtype=rdt)
    fh_np = W.fhat_gaussian(M, d, batch=B, dtype=cdt)
    gf_np = W.adjoint_input(N, batch=B, dtype=cdt)
    x = to_dev(x_np).requires_grad_(True)
    fh = to_dev(fh_np).requires_grad_(True)
    f = nfft_bandlimited(fh, x, plan)
    f.backward(to_dev(gf_np))
    op = oracle_plan(plan)
    assert rel_l2(to_host(x.grad), O.node_grad(op, fh_np, x_np, gf_np)) < tol
    assert rel_l2(to_host(fh.grad), O.adjoint(op, gf_np, x_np)) < (1e-12 if prec == "f64" else 1e-5)


def test_node_grad_central_differences():
    """d/dx of Re<g, f(x)> along random directions: central differences with
    h = 1e-4 / L and one Richardson step, all through the GPU FP64 path."""
    d, M, m, N = 2, 32, 6, 300
    plan = nb.Plan(d, M, 2.0, m, precision="f64")
    x_np = W.nodes_feasible(N, d, m, 2 * M, dtype=np.float64, seed=8)
    fh = to_dev(W.fhat_gaussian(M, d, dtype=np.complex128))
    g_np = W.adjoint_input(N, dtype=np.complex128)
    g = to_dev(g_np)
    plan.set_nodes(to_dev(x_np))
    gx = to_host(plan.node_grad(fh, g))
    v = W.fd_directions(N, d)

    def phi(xx):
        plan.set_nodes(to_dev(xx))
        return float(np.real(np.vdot(g_np, to_host(plan.forward(fh)))))

    def cd(h):
        return (phi(x_np + h * v) - phi(x_np - h * v)) / (2 * h)
    h = 1e-4 / plan.L[0]
    rich = (4 * cd(h / 2) - cd(h)) / 3
    exact = float(np.sum(gx * v))
    assert abs(rich - exact) <= 1e-7 * abs(exact)


def test_backward_after_other_nodes():
    """backward re-sets the plan's nodes when another forward intervened."""
    from paper_2502_07155_gb300.autograd import nfft_bandlimited
    plan = nb.Plan(2, 16, 2.0, 4, precision="f64")
    x1 = to_dev(W.nodes_uniform(50, 2, dtype=np.float64, seed=1)).requires_grad_(True)
    x2 = to_dev(W.nodes_uniform(70, 2, dtype=np.float64, seed=2))
    fh = to_dev(W.fhat_gaussian(16, 2, dtype=np.complex128)).requires_grad_(True)
    f1 = nfft_bandlimited(fh, x1, plan)
    nfft_bandlimited(fh.detach(), x2, plan)            # changes the plan's nodes
    f1.abs().pow(2).sum().backward()
    ref = nb.Plan(2, 16, 2.0, 4, precision="f64")
    x1b = x1.detach().clone().requires_grad_(True)
    fhb = fh.detach().clone().requires_grad_(True)
    nfft_bandlimited(fhb, x1b, ref).abs().pow(2).sum().backward()
    assert torch.allclose(x1.grad, x1b.grad) and torch.allclose(fh.grad, fhb.grad)
